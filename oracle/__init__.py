"""FP64 CPU oracle (test infrastructure only; never imported by the product path).

See fh_oracle for the statement of each step and the paper passage it follows.
"""
from .fh_oracle import *  # noqa: F401,F403
from .fh_oracle import (discretize, kress_weights, cfie_matrix, cfie_rhs, solve_density,  # noqa: F401
                        target_field, eta_w, window, window_centers, window_count,
                        window_spectra, full_band, synthesize, solve_all, target_fields, run)
