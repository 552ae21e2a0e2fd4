"""ORACLE — test infrastructure only.

A plain, slow, independent CPU implementation of what the GPU path computes: the loop
hafnian (three evaluators in lhaf_oracle.c) and the Gaussian-state algebra around it
(gbs.py). Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
it; the product package never does.
"""
