"""Plain CPU oracle for the SGM + scene-flow hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package.  It shares no code with the CUDA implementation.
"""
