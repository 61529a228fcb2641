"""CPU oracle for the GTQA hot path (TEST INFRASTRUCTURE ONLY).

Plain complex128 NumPy restatement of arXiv:2409.12240 plus an exact statevector
simulator used to pin it.  Imported only by tests/, by the smoke check in
__graft_entry__.py and by bench.py's CPU-baseline leg; the CUDA library never
imports or links anything from here.
"""
