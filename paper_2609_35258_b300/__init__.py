"""B300-native (sm_103a) hot path of MLVS-DUGKS behind the C ABI in include/mlvs.h.

``mlvs`` is the ctypes binding (same names as the C entry points); ``solver.Solver`` wraps a
workload description from ``workloads`` into create / set_velocity_levels / step / moments.
"""
