"""GB300-native (sm_103a) hot path of the master-slave PGA for unsupervised market
clustering (Hendricks, Gebbie & Wilcox, arXiv:1403.4099).

Submodules:
  synth    seeded synthetic inputs (no method arithmetic)
  gpga     ctypes binding of the C-ABI library libgpga.so (cluster_corr, ga_score,
           ga_init, ga_step, ga_best, ...); fails loudly if the library is missing
  metrics  adjusted Rand index for recovery measurements
  build    nvcc build of libgpga.so for sm_103a
"""
