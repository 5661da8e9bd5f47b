"""SAC-family 2D ideal-MHD step on B300 (arXiv 1710.06423)."""
