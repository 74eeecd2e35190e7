// Kernel instantiations: double, grid sizes X(16) X(32) X(64) X(128) X(256) X(512).
#define TTSH_T double
#define TTSH_REGISTRY ops_f64_small
#define TTSH_SIZES X(16) X(32) X(64) X(128) X(256) X(512)
#include "ttsh_ops_impl.cuh"
