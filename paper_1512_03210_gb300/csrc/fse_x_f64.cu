// fse_x_f64.cu -- x-pass instantiations for double.
#include "fse_launch.cuh"

namespace fse {
template cudaError_t launch_xpass<double>(int, int, const XArgs&, const void*, const void*, cudaStream_t);
template int xpass_ncol<double>(int);
template int xpass_ncol_x2<double>(int);
}  // namespace fse
