"""dagrt: GB300-native batched evaluation of the makespan bound of "Exploiting
Dependency and Parallelism: Real-Time Scheduling and Analysis for GPU Tasks".

Submodules:
  workloads -- seeded synthetic DAG batches and candidate allocations (inputs only)
  build     -- nvcc build of libdagrt.so (sm_103a)
  dagrt     -- ctypes binding of the C ABI declared in include/dagrt.h
"""
