// Persistent batched stepper, double domains.
#define TTSH_T double
#define TTSH_PERSIST_REGISTRY persist_f64
#include "ttsh_persist_impl.cuh"
