"""CPU FP64 oracle of the ladder dual-fermion loop: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs may
import this package; the product path (paper_1507_00895_gb300) never does.
"""
