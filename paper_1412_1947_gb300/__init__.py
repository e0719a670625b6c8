"""GB300-native two-level sampling-based clustering (landmark peel + batched Lloyd)."""
