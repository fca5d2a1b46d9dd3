"""GB300-native batched exact matching of DNA queries over suffix arrays.

The compute path lives in the CUDA library ``libsa.so`` (C ABI declared in
``include/sa.h``); :mod:`paper_1303_3692_gb300.sa` is its thin ctypes binding.
:mod:`paper_1303_3692_gb300.datagen` draws the seeded synthetic workloads.
"""
