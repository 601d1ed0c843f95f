"""GB300-native multidimensional phase-shift sparse FFT (partial unwrapping, tilted lines)."""
