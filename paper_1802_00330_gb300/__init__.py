"""GB300-native interval branch-and-bound + Hansen-Sengupta solver (binding package)."""
