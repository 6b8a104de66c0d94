// transforms_f32.cu -- explicit instantiations of the transform kernels
// (transforms.cuh) in FP32 arithmetic; one translation unit per
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
RSFDE_TOEP_COLS(float, float, float)
RSFDE_TOEP_COLS(float, double, float)
RSFDE_TOEP_COLS(float, float, double)
RSFDE_TOEP_COLS(float, double, double)
RSFDE_TOEP_ROWS(float, double)
RSFDE_TOEP_ROWS(float, float)
RSFDE_DST_ROWS(float, double, float)
RSFDE_DST_ROWS(float, df, float)
RSFDE_DST_ROWS(float, float, float)
template void launch_precond_cols<float>(const float*, float*, float*, int, int, const AxisTables<float>&,
                                         const float*, double, const int*, cudaStream_t);
template void launch_precond_rows<float, float>(const float*, const float*, const uint8_t*, float*, int, int,
                                                const AxisTables<float>&, const int*, cudaStream_t);
template void launch_precond_rows<float, double>(const float*, const float*, const uint8_t*, double*, int, int,
                                                 const AxisTables<float>&, const int*, cudaStream_t);

#define RSFDE_OP_MULTI(T, Tz, Tv) \
  template void launch_operator_multi<T, Tz, Tv>(const BatchInst*, const MultiGrid&, const MultiGrid&, int, cudaStream_t);
RSFDE_OP_MULTI(float, float, double)
RSFDE_OP_MULTI(float, float, float)
template void launch_precond_multi<float, float, double>(const BatchInst*, const MultiGrid&, const MultiGrid&,
                                                         const MultiGrid&, int, cudaStream_t);
template void launch_precond_multi<float, float, float>(const BatchInst*, const MultiGrid&, const MultiGrid&,
                                                        const MultiGrid&, int, cudaStream_t);

}  // namespace rsfde
