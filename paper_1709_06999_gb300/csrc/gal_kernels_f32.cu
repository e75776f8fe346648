// Single-precision instantiation of the kernels (FP32 bulk arithmetic,
// float-float index and phase arguments, FP64 reduction).
#include "gal_kernels.cuh"
template struct gal::Launch<float>;
