"""B300-native (sm_103a) VOLKS2 cross-spectrum single-pulse search."""
