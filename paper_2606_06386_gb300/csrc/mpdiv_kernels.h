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
// the plain division kernel with 128 registers per thread (mpdiv_k{4,8,16}r.cu):
// 4 warps x 4 blocks, 8 warps x 2 blocks, 16 warps x 1 block per SM
void* mp_kernel_w4_wide();
void* mp_kernel_w8_wide();
void* mp_kernel_w16_wide();
// the plain division kernel over a ragged batch's item list (64 registers),
// mpdiv_l{1,2,4,8,16,32}.cu: the class form of mpdiv_batch_ragged
void* mp_kernel_list(int warps);
void* mp_kernel_list1();
void* mp_kernel_list2();
void* mp_kernel_list4();
void* mp_kernel_list8();
void* mp_kernel_list16();
void* mp_kernel_list32();
void* mp_kernel_persistent(int warps);  // 8 (warps <= 8) or 16 warps per block
void* mp_kernel_persistent8();          // mpdiv_p.cu
void* mp_kernel_persistent16();         // mpdiv_p16.cu
void* mp_kernel_w16_queue(int kind);    // mpdiv_q.cu: MP_K_RAGGED and MP_K_SHINV
void* mp_kernel_prim(int warps);        // mpdiv_t.cu: the primitive test kernel (1, 2, 4, 8, 16, 32 warps)
// mpdiv_t.cu: the multiply-pipe microbenchmark (kind 0: digit products, 1:
// 32-bit multiply-adds) for 256-thread blocks; *ops_per_round per thread and round
void* mp_kernel_peak(int kind, int* ops_per_round, int* smem_bytes, int* blocks_per_sm);
// kernels whose full products may use the number-theoretic transform
void* mp_kernel_ntt_uniform(int warps);  // mpdiv_n.cu: 4, 8, 16 or 32 warps (ntt_kernel_warps)
void* mp_kernel_ntt_mul(int warps);      // mpdiv_n.cu: the multiplication cost unit, 4, 8, 16 or 32 warps
void* mp_kernel_ntt_uniform8();          // mpdiv_n8.cu
void* mp_kernel_ntt_uniform16();         // mpdiv_n16.cu
void* mp_kernel_ntt_uniform32();         // mpdiv_n32.cu
void* mp_kernel_ntt_queue(int kind);     // mpdiv_n2.cu: MP_K_RAGGED and MP_K_SHINV, 16 warps
void* mp_kernel_ntt_shinv();             // mpdiv_n3.cu
