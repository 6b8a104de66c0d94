// transforms_f64.cu -- explicit instantiations of the transform kernels
// (transforms.cuh) in FP64 arithmetic; one translation unit per
// arithmetic type so that the library's objects compile in parallel.
#include "transforms.cuh"

namespace rsfde {

#define RSFDE_TOEP_COLS(T, Tin, Tout)                                                                           \
  template void launch_toeplitz_cols<T, Tin, Tout>(int, const Tin*, void*, const uint8_t*, double, const double*, \
                                                   Tout*, int, int, const AxisTables<T>&, const int*, double*,    \
                                                   SolverState*, cudaStream_t);
#define RSFDE_TOEP_ROWS(T, Tin) \
  template void launch_toeplitz_rows<T, Tin>(const Tin*, void*, const uint8_t*, double, int, int,   \
                                              const AxisTables<T>&, const int*, cudaStream_t);
#define RSFDE_DST_ROWS(T, Tin, Tout)                                                                        \
  template void launch_dst_rows<T, Tin, Tout>(const Tin*, const double*, Tout*, int, int, const AxisTables<T>&, \
                                              const int*, cudaStream_t);
RSFDE_TOEP_COLS(double, double, double)
RSFDE_TOEP_COLS(double, float, double)
RSFDE_TOEP_COLS(double, double, df)
RSFDE_TOEP_COLS(double, double, float)
RSFDE_TOEP_ROWS(double, double)
RSFDE_TOEP_ROWS(double, float)
RSFDE_DST_ROWS(double, double, double)
RSFDE_DST_ROWS(double, double, float)
RSFDE_DST_ROWS(double, df, double)
RSFDE_DST_ROWS(double, float, double)
template void launch_dst_cols<double, double, double>(const double*, double*, int, int, const AxisTables<double>&,
                                                      cudaStream_t);
template void launch_precond_cols<double>(const double*, double*, double*, int, int, const AxisTables<double>&,
                                          const double*, double, const int*, cudaStream_t);
template void launch_precond_rows<double, double>(const double*, const double*, const uint8_t*, double*, int, int,
                                                  const AxisTables<double>&, const int*, cudaStream_t);
template void launch_precond_rows<double, float>(const double*, const double*, const uint8_t*, float*, int, int,
                                                 const AxisTables<double>&, const int*, cudaStream_t);

template void launch_residual_multi<double, double>(const BatchInst*, const MultiGrid&, const MultiGrid&,
                                                   cudaStream_t);
template void launch_residual_multi<double, float>(const BatchInst*, const MultiGrid&, const MultiGrid&, cudaStream_t);

}  // namespace rsfde
