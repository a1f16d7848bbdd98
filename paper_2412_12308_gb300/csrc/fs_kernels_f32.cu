// FP32 instantiation of the kernels and launchers.
#include "fs_kernels.cuh"
#include "fs_tma.cuh"
namespace fs {
__device__ int g_fs_dev_error = 0;
template struct Launch<float>;
}
