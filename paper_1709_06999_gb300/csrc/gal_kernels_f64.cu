// Double-precision instantiation of the kernels.
#include "gal_kernels.cuh"
template struct gal::Launch<double>;
