"""GB300-native Fireflies hot path (binding is loaded lazily)."""
