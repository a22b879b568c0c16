"""CPU oracle for homogeneous diffusion inpainting (TEST INFRASTRUCTURE ONLY).

This package is the slow, plainly written FP64 reference that the CUDA path is
checked against.  Only the test suite, the smoke check and the CPU-baseline leg
of the benchmark may import it; the library itself never calls it and has no
CPU fallback.  It shares no code with the CUDA path: the only common module is
``synth`` (seeded inputs, no solver arithmetic).

Modules
  inpaint_ref  -- the problem (Sec. 2, Eq. eq:homdiff / eq:ls): Laplacian with
                  reflecting boundaries, A = C - (I-C)L, b = Cf, residuals, the
                  relative-residual stop measure, and the exact solution by a
                  sparse direct solve.
  cg           -- plain FP64 conjugate gradients on the unknown pixels (C with
                  OpenMP, ``cg_ref.c``) for frames too large for the direct solve.
  oras_ref     -- the restricted additive Schwarz steps of Sec. 3-4 in the
                  paper's order: block layout, restriction R_i, partition of
                  unity D_i, local problem R_i A R_i^T with the optimised
                  (Robin) interface condition, local CG, restricted add-back;
                  dyadic mask/value subsampling and the coarse-to-fine
                  prolongation of the multilevel variant.
"""
