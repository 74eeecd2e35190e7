// Persistent batched stepper, float domains.
#define TTSH_T float
#define TTSH_PERSIST_REGISTRY persist_f32
#include "ttsh_persist_impl.cuh"
