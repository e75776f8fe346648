// Batched passes, float32 instantiation.
#include "gal_batch.cuh"

template struct gal::BatchLaunch<float>;
