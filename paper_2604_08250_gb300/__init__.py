"""GB300-native swap Monte Carlo on BCC alloys (SMC-X / SMC-AI hot path).

Submodules: ``smc`` (ctypes binding of libsmc.so), ``inputs`` (seeded
synthetic workloads), ``build`` (compiles libsmc.so for sm_103a).
"""
