// Instantiates the work units for one element type and register tile size,
// and the RK4 pass kernels of the same tile (fs_rk4.cuh).
// Compiled once per (FS_T, FS_E) pair by the build, as relocatable device code.
#include "fs_rk4.cuh"
#include "fs_units.cuh"

#ifndef FS_T
#error "FS_T (float or double) must be defined"
#endif
#ifndef FS_E
#error "FS_E (register tile size) must be defined"
#endif

// expand FS_T / FS_E before token pasting
#define FS_UNIT_DEF_X(T, E) FS_UNIT_DEF(T, E)
#define FS_RK4_DEF_X(T, E) FS_RK4_DEF(T, E)

namespace fs {
FS_UNIT_DEF_X(FS_T, FS_E)
FS_RK4_DEF_X(FS_T, FS_E)
}
