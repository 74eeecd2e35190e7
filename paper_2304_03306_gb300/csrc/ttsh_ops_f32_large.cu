// Kernel instantiations: float, grid sizes X(1024) X(2048) X(4096) X(8192).
#define TTSH_T float
#define TTSH_REGISTRY ops_f32_large
#define TTSH_SIZES X(1024) X(2048) X(4096) X(8192)
#include "ttsh_ops_impl.cuh"
