"""FP64 CPU oracle of the JDE detect-and-track path (test infrastructure only).

This package is the plain, slow reference that the CUDA library is checked
against.  It is imported only by ``tests/``, by ``__graft_entry__.smoke()`` and
by the CPU-baseline leg of ``bench.py``; the product path (``libjde`` and its
Python binding) never imports, links or runs it, and it shares no code with
that path.  Inputs come from the ``synth`` generators.

Modules and the passages they follow:

* ``network``     - letterbox, DarkNet-53 + FPN + detection/embedding heads
                    (Sec. 3.1; architecture readings for the unstated layer
                    table, weights and letterbox geometry).
* ``postprocess`` - anchor decode, confidence filter, greedy NMS, embedding
                    normalisation (Sec. 3.2 and Appendix A, first three steps).
* ``tracker``     - Kalman predict/update, cosine cost, motion gating,
                    Hungarian assignment, track lifecycle (Sec. 3 "Location
                    Estimation" / "Association" and Appendix A, remaining steps).

Every floating-point step runs in float64.  The network as a whole is
"parity unpinned" against the paper: the paper prints no layer table, no
trained weights and no worked numeric example, so each operation is pinned
separately (brute force, library cross-checks, closed forms) but the assembled
network can only be pinned by construction (layer count, parameters, FLOPs).
"""
