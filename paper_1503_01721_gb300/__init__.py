"""GB300-native hot path of column-generation VMAT optimisation (arXiv:1503.01721)."""
