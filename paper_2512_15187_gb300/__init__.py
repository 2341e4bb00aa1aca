"""Probabilistic Inclusion Depth (PID) on GB300 (sm_103a).

Public surface:
  binding   ctypes mirror of the C ABI in include/pid.h (pid_* functions, Handle)
  synth     seeded synthetic ensembles shaped like the paper's workloads
  build     compiles csrc/ into the in-tree libpid.so
"""
__all__ = ["binding", "synth", "build"]
