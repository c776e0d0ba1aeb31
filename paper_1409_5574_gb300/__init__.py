"""prad: GB300-native synchrotron photon emission for particle pushers.

The hot path of arXiv:1409.5574 (field gather, Boris push, H_eff and omega_c,
Monte-Carlo emission with the S(x) noise-reduction proposal, photon append and
the emitted-energy vs Landau-Lifshitz ledger) runs in hand-written sm_103a CUDA
kernels behind the C ABI declared in ``include/prad.h``. ``prad`` is the thin
ctypes binding; nothing is loaded at import time.
"""
__all__ = ["prad", "workloads"]
