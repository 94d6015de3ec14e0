"""GB300-native Wolstenholme/Vandiver residue search (lazy; see wv.py)."""
