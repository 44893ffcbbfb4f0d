"""FP64 CPU oracle of the hierarchically tiled 3DGS render path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or runs anything here; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.  The
oracle shares no code, constants, tables or helpers with the CUDA path.

What it computes is the plain 3D Gaussian Splatting forward model the paper
renders exactly (abstract; Sec. 3.4, Eq. 1 "compose"), in float64, from the
float32 scene parameters:

  * ``project``   - per-gaussian EWA projection + SH colour (Sec. 4.2; the
                    formulas are the original 3DGS ones, which the paper
                    defers to as "standard").
  * ``composite`` - per-pixel support test, alpha and ordered front-to-back
                    compositing with per-pixel termination (Sec. 3.4).
  * ``binning``   - the discrete stages on float32 records: rect binning over
                    render or macro tiles (Sec. 3.2, 4.3), the (depth key, id)
                    segment order (Sec. 3.3, 4.4) and the fixed-size batch
                    split (Sec. 3.1).
  * ``batched``   - the macro-tile/batch decomposition with Eq. 1 merging and
                    exact-termination replay, used to pin the invariance
                    "any macro shape or batch cap gives the same image".
  * ``grad``      - analytic FP64 gradient of 0.5*||C - C_target||^2.
  * ``train``     - the L2 loss and the Adam step of the differentiable path.
  * ``sh_codec``  - the 32-byte packed SH representation (Sec. 4.2).
  * ``order``     - the spatial (Morton) storage order of a scene (a memory
                    layout outside the paper's method).

Every function names the passage it follows; readings of silent or
ambiguous passages are listed in the repository's design notes.
"""
