"""GB300-native ST-HOSVD Tucker compression (TuckerMPI hot path)."""
