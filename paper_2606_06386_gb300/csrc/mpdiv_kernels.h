// Getters for the kernel instantiations of each block size (mpdiv_k*.cu): the
// plain division and multiplication kernels at every size; the queue, test and
// persistent kernels where noted.
#pragma once

enum { MP_K_UNIFORM = 0, MP_K_RAGGED = 1, MP_K_SHINV = 2, MP_K_PERSIST = 3, MP_K_MUL = 4 };

void* mp_kernel_w1(int kind);
void* mp_kernel_w2(int kind);
void* mp_kernel_w4(int kind);
void* mp_kernel_w8(int kind);  // also the self-splitting persistent kernel (8 -> 4 -> 2 warps)
void* mp_kernel_w16(int kind);  // also the self-splitting persistent kernel (16 -> 8 -> 4 warps),
                                // the one-block-per-item queue kernel and the shifted-inverse test entry
void* mp_kernel_w32(int kind);
void* mp_kernel_persistent(int warps);  // 8 (warps <= 8) or 16 warps per block
void* mp_kernel_persistent8();          // mpdiv_p.cu
void* mp_kernel_persistent16();         // mpdiv_p16.cu
void* mp_kernel_w16_queue(int kind);    // mpdiv_q.cu: MP_K_RAGGED and MP_K_SHINV
void* mp_kernel_prim(int warps);        // mpdiv_t.cu: the primitive test kernel (1, 2, 4, 8, 16, 32 warps)
