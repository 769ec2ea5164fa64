// fse_col_f32.cu -- column-pass instantiations for float.
#include "fse_launch.cuh"

namespace fse {
template cudaError_t launch_colpass<float>(int, int, const ColArgs&, const MulArgs&, const void*, cudaStream_t);
template int colpass_ncol<float>(int);
}  // namespace fse
