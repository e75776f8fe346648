// Batched passes, float64 instantiation.
#include "gal_batch.cuh"

template struct gal::BatchLaunch<double>;
