"""GB300-native render path of 4D Gaussian Splatting (arXiv 2412.20720)."""
