"""FP64 CPU oracle of the masked 4D Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path (the CUDA library and its Python binding) never
does, and shares no code with it.

Parity status per function (what pins each one is in tests/test_oracle_pins.py):
  keyframe_pair, active_from_masks ........ pinned (hand-built key-frame cases, all-ones /
                                            all-zeros masks)
  rotation_4d, covariance_4d .............. pinned (orthogonality, det = +1, identity,
                                            independent Hamilton-product construction)
  condition_on_time (Eq. 1, Eq. 3) ........ pinned (Schur complement of the precision
                                            matrix, density maximisation, finite differences)
  sh_basis ................................ pinned (scipy complex spherical harmonics,
                                            closed-form degree-1 colours of known view
                                            directions)
  preprocess / tile_lists / blend_tile .... pinned (NumPy brute-force renderer, single- and
                                            two-Gaussian closed forms, zero space-time
                                            correlation reducing to a static 3D splat,
                                            tile-rectangle brute force, a hand-built
                                            indefinite conic for the power > 0 skip)
  gradients ............................... pinned (float64 central finite differences)
  variation_scores, keep_set .............. pinned (weight identity, factor range, gamma
                                            range, permutation invariance, R1 = R2 at one t)
  score variants of the ablation (Table 4) . pinned (each rendered variant against the spatial
  temporal_first_derivative                 score, Sigma_t = exp(2 l_t) at identity rotations,
                                            the temporal-only score's independence of the
                                            views, finite differences for p^(1))
tests/test_oracle_mutations.py plants plausible mistakes in these functions and checks that
the pins catch each one.
No values printed in the paper can pin any of them: the paper gives no worked example, so
agreement with the paper's own numbers is "parity unpinned" for every function.
"""
from .fdgs_oracle import *  # noqa: F401,F403
from .fdgs_oracle import (ALPHA_MAX, ALPHA_MIN, T_STOP, TILE, Params, active_from_masks,  # noqa
                          blend_tile, condition_on_time, covariance_4d, gradients, keep_set,
                          keyframe_pair, preprocess, render, render_image, rotation_4d,
                          sh_basis, temporal_first_derivative, temporal_second_derivative,
                          tile_list, tile_lists, variation_factor, variation_scores,
                          volume_gamma, SCORE_VARIANTS)
