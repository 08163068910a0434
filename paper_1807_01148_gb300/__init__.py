"""GB300-native traffic microsimulation hot path (Waddell et al., Sec. 6)."""
