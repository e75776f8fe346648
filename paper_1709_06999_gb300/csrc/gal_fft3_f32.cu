// Compile-time-length FFT passes, float32 instantiations.
#include "gal_fft3_launch.cuh"
namespace gal {
template cudaError_t row_fft3<float>(const float*, const float*, const SweepParams&, int,
                                     const void*, void*, const double*, double, int*, const float*, cudaStream_t, int);
template cudaError_t col_fft3<float>(const void*, void*, int, const void*, const double*, double,
                                   int, bool, cudaStream_t, int);
}  // namespace gal
