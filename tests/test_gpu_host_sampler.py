"""The host sampler's parity tests, run on the GPU's host (marked gpu).

vndf_cpu_sample is timed for the paper's CPU protocol (Sec. 4) on the host that
drives the GPU, an AArch64 machine where it is built for NEON.  The same parity
checks as tests/test_cpu_sampler.py (FP64 oracle, stored 50-digit rows, thread
and isotropy independence, the double-precision recomputation) run here
under the gpu marker so that the GPU pass checks that build where it is timed.
"""
import pytest

from test_cpu_sampler import (  # noqa: F401  (the fixture and the tests are collected here again)
    test_cpu_cap_extended_matches_oracle, test_cpu_cap_matches_oracle, test_cpu_domain_fallback_and_errors,
    test_cpu_precise_meets_the_flat_bounds, test_cpu_precise_on_stored_samples, test_cpu_precise_on_wide_inputs,
    test_cpu_prior_matches_oracle, test_cpu_results_independent_of_threads_and_isotropy,
    test_cpu_sampler_on_stored_samples, v)

pytestmark = pytest.mark.gpu
