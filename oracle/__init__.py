"""FP64 CPU oracle (test infrastructure).  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs may import it; the product path never does."""
