"""GB300-native batched unfolded ISTA / Step-LISTA / Oracle-ISTA (arXiv 1905.11071)."""
