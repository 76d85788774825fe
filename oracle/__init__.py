"""FP64 CPU oracle for the randomized DOT hot path (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
package; the library itself never does.
"""
