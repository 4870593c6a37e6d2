"""GPU greedy kNN-cost point-cloud decimation for GB300 (sm_103a).

Method: Comino-Trinidad, Chica, Andujar, "Revisiting Poisson-disk Subsampling
for Massive Point Cloud Decimation" (arXiv 2311.17604).

  synth   seeded synthetic LiDAR scans (inputs only)
  build   compiles libpd.so in-tree with nvcc
  pd      ctypes binding of the C ABI in include/pd.h
"""
