"""GB300-native on-the-fly property library (arXiv 2503.07526).

Lennard-Jones MD on one GPU with the system stress tensor, heat flux and
multiple-tau correlators (stress, heat flux, per-atom velocity) computed
while the simulation runs, plus Green-Kubo integrals, and a learned
Green-Kubo tail (a tensor-core network that predicts converged transport
coefficients from a short run).  The compute lives in ``libotfmd.so`` (C ABI
in ``include/otf_md.h`` and ``include/gk_tail.h``); this package only
marshals arguments.
"""
from ._lib import (  # noqa: F401
    EXPORTS,
    MD_CORR_HEATFLUX,
    MD_CORR_MASSFLUX,
    MD_CORR_STRESS,
    MD_CORR_VACF,
    MD_K_NAMES,
    MD_MEM_DEVICE,
    MD_MEM_HOST,
    MD_PAIR_CELLS,
    MD_PAIR_TILES,
    MD_PAIR_VERLET,
    MD_POT_BUCK_EWALD,
    MD_POT_LJ,
    KE_EV_ANGSTROM,
    MD_PREC_FP64,
    MD_PREC_MIXED,
    MLP,
    Corr,
    MdError,
    System,
    gk_integrate,
    gk_tail_box,
    gk_tail_choose,
    gk_tail_features,
    gk_tail_rms_rel,
    lib,
    fp32_peak,
    make_params,
    observables_noalloc,
)
