"""GB300-native batched trust-region Newton (TRON) and component ADMM (arXiv 2106.14995)."""
