"""GB300 (sm_103a) ABC rejection sampling of the six-compartment stochastic
COVID-19 model (Kulkarni, Krell, Nabarro, Moritz 2020).

The computation runs in the CUDA library ``libabc_gb300.so`` behind the C ABI
of ``include/abc_gb300.h``; ``binding`` marshals arguments to it.
"""
from .binding import (ABC_EXACT, ABC_FAST, ABC_MAX_REGIONS, ABC_VARIANCE_LITERAL, ABC_NOALLOC_T_MAX, ABC_T_MAX,  # noqa: F401
                      PAPER_HI, PAPER_LO, AbcError, Flow, Observed, Plan, abc_distances, abc_kth_smallest, abc_select_below, abc_sample_quantile,
                      abc_last_simulated_days, abc_pmc_propose, abc_pmc_run, abc_pmc_weights,
                      abc_project, abc_sample, abc_sample_async, abc_sample_noalloc, abc_sample_until, abc_simulate,
                      abc_smc_run, abc_smc_run_regions, abc_step, abc_strerror, abc_version, load, prior_box)
