// fse_x_f32.cu -- x-pass instantiations for float.
#include "fse_launch.cuh"

namespace fse {
template cudaError_t launch_xpass<float>(int, int, const XArgs&, const void*, const void*, cudaStream_t);
template int xpass_ncol<float>(int);
template int xpass_ncol_x2<float>(int);
}  // namespace fse
