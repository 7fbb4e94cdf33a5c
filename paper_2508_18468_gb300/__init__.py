"""GB300-native monitored free-fermion trajectories (arXiv 2508.18468).

``fm`` binds the CUDA library ``libfm.so`` (C ABI in ``include/fm.h``);
``build`` compiles it for sm_103a; ``workloads`` holds the seeded synthetic
workload definitions.
"""
