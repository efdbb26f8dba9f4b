"""CPU FP64 oracle for the ANKH hot path.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py may import anything in this
package.  It shares no code with the CUDA path.
"""
