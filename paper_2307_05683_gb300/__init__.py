"""GB300-native FP64 ensemble Wisdom-Holman integrator (WHFast512's timestep).

The integrator itself lives in a CUDA C-ABI library (libwhg, built from
csrc/ for sm_103a); `paper_2307_05683_gb300.whg` is its thin Python binding.
`paper_2307_05683_gb300.inputs` makes seeded synthetic planetary ensembles.
Submodules load lazily so that input generation works on machines without
the library; every integrator call fails loudly if the library is missing.
"""
__all__ = ["inputs", "whg"]
