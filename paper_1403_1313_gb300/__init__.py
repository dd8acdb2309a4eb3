"""GB300 Skip-Brute-Force planted (l,d) motif search (placeholder, filled in below)."""
