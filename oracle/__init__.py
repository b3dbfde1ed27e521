"""FP64 CPU oracle for the staggered-grid pressure projection (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may import
this package.  The product path (paper_2609_19130_gb300) never does.
"""
