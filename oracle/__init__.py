"""FP64 CPU oracle for the 3DGS-LM hot path (arXiv 2409.12892).

TEST INFRASTRUCTURE. This package is the slow, plain reference the CUDA path is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. It
shares no code with the CUDA library and imports nothing from the product
package; its inputs come from ``synth`` (seeded random numbers only).

Everything is float64 NumPy. Each function cites the passage of the paper it
follows. Where the paper defers to the 3DGS rasterizer for a constant or
convention, the reading is stated in ``oracle.conventions``.

Modules
    conventions  rasterizer constants and conventions (paper silent; see docstring)
    ad           forward-mode dual numbers (exact first derivatives)
    sh           real spherical harmonics of degree <= 3
    projection   Gaussian -> 2D splat, with its exact 9 x 59 Jacobian dy/dx
    raster       tile-ordered front-to-back alpha blending, per-pixel records
    jacobian     J p, J^T u, diag(J^T J), explicit sparse J (per-pixel chain rule)
    solver       Algorithm 1 (PCG), the subset weighted mean, the LM step
    mlp          per-Gaussian MLP of the learned diagonal preconditioner
"""
