// FP64 instantiation of the kernels and launchers.
#include "fs_kernels.cuh"
namespace fs {
template struct Launch<double>;
}
