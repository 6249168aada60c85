"""GB300-native SINNAMON: streaming sparse maximum inner product search."""
