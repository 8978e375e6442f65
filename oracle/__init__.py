"""CPU oracle for the Reed-Solomon path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs may import this package.
"""
