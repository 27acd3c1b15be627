"""Oracle — test infrastructure only.

A plain, slow, FP64 CPU statement of what the butterfly path computes:
  direct.py / direct.c  the sparse Fourier transform by its definition (eq. 1.1) and its
                        adjoint, summed term by term;
  butterfly.py          the butterfly algorithm of Sec. 2.2, steps 1-4, in the paper's
                        order and notation, with M and E built from grid coordinates.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import it.  It
shares no code with the CUDA path and imports nothing from it.
"""
