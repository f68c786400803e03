"""SyMBA hot path on GB300 (arXiv:2304.07325)."""
