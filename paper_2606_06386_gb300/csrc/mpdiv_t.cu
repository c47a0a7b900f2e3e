// The group-primitive test kernel for every block size, in a translation unit
// of its own.
#include "mp_kernels.cuh"
#include "mpdiv_kernels.h"

void* mp_kernel_prim(int warps) {
  switch (warps) {
    case 1: return (void*)mp::k_prim<1, 32>;
    case 2: return (void*)mp::k_prim<2, 16>;
    case 4: return (void*)mp::k_prim<4, 8>;
    case 8: return (void*)mp::k_prim<8, 4>;
    case 16: return (void*)mp::k_prim<16, 2>;
    default: return (void*)mp::k_prim<32, 1>;
  }
}
