"""GB300-native homogeneous-embedding IPM (CuClarabel-style) per-iteration device step."""
