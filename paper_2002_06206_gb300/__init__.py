"""GB300 (sm_103a) implementation of the topology-free immersed-boundary LES step of Onishi &
Tsubokura (arXiv 2002.06206): CUDA kernels behind the C ABI of include/ibmles.h, and a thin Python
binding (ibmles) over it.  The build module compiles libibmles.so in-tree with nvcc."""
