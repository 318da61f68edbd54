"""GB300-native DPD time step with phase-field no-slip walls (Xu & Meakin, arXiv:1807.09896).

* ``dpd``     -- ctypes binding of the C ABI in ``include/dpd.h`` (``libdpd.so``);
* ``inputs``  -- seeded synthetic workloads (channels, bulk boxes, sphere packs);
* ``_build``  -- nvcc build of ``libdpd.so`` for sm_103a.

The CUDA library is loaded on first use, not at import, so the input generators
can be imported on machines without a GPU.
"""

__all__ = ["dpd", "inputs"]
