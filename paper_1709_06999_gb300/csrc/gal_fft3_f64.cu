// Compile-time-length FFT passes, float64 instantiations.
#include "gal_fft3_launch.cuh"
namespace gal {
template cudaError_t row_fft3<double>(const double*, const double*, const SweepParams&, int,
                                      const void*, void*, const double*, double, int*,
                                      const double*, cudaStream_t, int);
template cudaError_t col_fft3<double>(const void*, void*, int, const void*, const double*, double,
                                   int, bool, cudaStream_t, int);
}  // namespace gal
