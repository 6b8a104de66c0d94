// transforms_df_a.cu -- explicit instantiations of the transform kernels
// (transforms.cuh) in double-FP32 (operator passes) arithmetic; one translation unit per
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
RSFDE_TOEP_COLS(df, float, double)
RSFDE_TOEP_COLS(df, float, df)
RSFDE_TOEP_ROWS(df, double)
RSFDE_TOEP_ROWS(df, float)


}  // namespace rsfde
