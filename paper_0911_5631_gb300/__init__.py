"""GB300-native soft-sphere molecular dynamics (placeholder; binding added later)."""
