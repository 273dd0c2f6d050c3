"""pmshrink: the shrinking-domain particle-mesh step (Llinares 2017,
arXiv:1709.04703) on one GB300, as hand-written sm_103a CUDA behind a C ABI
(include/pmshrink.h).

Importing the package loads nothing; ``Sim``, ``power_spectrum`` and
``deposit`` load libpmshrink.so on first use and raise if it is missing.
``ics`` (seeded inputs) needs neither torch nor CUDA.
"""
__all__ = ["Sim", "power_spectrum", "deposit", "pack", "unpack"]


def __getattr__(name):
    if name in __all__:
        from . import sim
        return getattr(sim, name)
    raise AttributeError(name)
