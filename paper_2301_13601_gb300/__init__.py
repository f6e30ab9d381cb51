"""GB300-native qubit lattice algorithm (QLA) for 2D Maxwell in diagonal-tensor dielectrics."""
