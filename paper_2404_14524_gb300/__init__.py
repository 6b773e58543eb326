"""GB300-native Nys-IP-PMM normal-equations solve (arxiv 2404.14524)."""
