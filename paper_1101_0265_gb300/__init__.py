"""GB300-native recursive density-matrix purification (libpurify)."""
