"""GB300-native yarn BYSDF (eval / sample / pdf / backward) behind a C-ABI library."""
