"""Plain FP64 CPU oracle for the per-sample PEPS contraction of PEPS++.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or
run anything in this package. The product path (the CUDA library and its
Python binding) never imports it and shares no code with it.

Every function follows a passage of the paper (He et al., "PEPS++: Towards
Extreme-scale Simulations of Strongly Correlated Quantum Many-particle Models
on Sunway TaihuLight", arXiv:1806.03761) and says which. Where the paper is
silent the reading taken is stated in the function's docstring.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against brute-force contraction, exact diagonalisation, closed forms, finite
differences, published Philox known-answer vectors or exact invariants.  In
the truncated regime (D_c below the exact bond dimension) the compression is
pinned against sequential truncated SVDs of the exact state vector (the
tensor-train SVD), and the evaluation on truncated environments through
invariants that hold at any D_c (the strip-local ratio and log-derivative
definitions, sum_T T Delta = 1 per site).
"""
from .peps import (  # noqa: F401
    bond_list, site_tensor, BMPS, compress, upper_envs, lower_envs,
    Strip1, Strip2, evaluate, evaluate_batch, gradient, go_step, amplitude,
)
from .philox import philox4x32_10, uniform53, uniform_open53  # noqa: F401
from .sampler import init_config, metropolis_sweep, sample_chains  # noqa: F401
from .correlations import (  # noqa: F401
    exchange_ratios, local_correlations, bulk_sites, structure_factor, centre_site,
)
