// fse_col_f64.cu -- column-pass instantiations for double.
#include "fse_launch.cuh"

namespace fse {
template cudaError_t launch_colpass<double>(int, int, const ColArgs&, const MulArgs&, const void*, cudaStream_t);
template int colpass_ncol<double>(int);
}  // namespace fse
