"""GB300-native non-polynomial (RBF-perturbed) ENO/WENO finite-volume solver (arXiv 1602.00182).

The compute path is the CUDA library ``libnpweno.so`` (C ABI, ``include/npweno.h``);
``paper_1602_00182_gb300.npweno`` is its thin ctypes binding.  ``inputs`` builds the seeded
synthetic workloads.
"""
