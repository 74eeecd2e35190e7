// Kernel instantiations: double, grid sizes X(1024) X(2048) X(4096).
#define TTSH_T double
#define TTSH_REGISTRY ops_f64_large
#define TTSH_SIZES X(1024) X(2048) X(4096)
#include "ttsh_ops_impl.cuh"
