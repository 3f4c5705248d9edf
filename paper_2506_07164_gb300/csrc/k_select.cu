// Top-N per level: keep the n_l best NMS survivors of each (frame, level)
// image in rank order -- Harris key descending, then y ascending, then x
// ascending (Harris "screens" the FAST points, Sec. 1 and Sec. 3.2).
//
// One block per image.  Each candidate has a unique 96-bit rank word
//   R = (key ^ 2^63) << 32 | ~((y << 16) | x),
// larger R = better rank.  An MSB-first radix select over 8-bit digits of R
// (one shared-memory histogram per pass) fixes, digit by digit, the prefix
// of the n_l-th largest R; it stops as soon as every candidate that shares
// the fixed prefix is needed.  The selected candidates are gathered into
// shared memory and bitonic-sorted by R, descending.
#include <cuda_runtime.h>

#include "of_internal.h"

namespace ofk {

struct SelState {
    uint64_t pre_hi, msk_hi;
    uint32_t pre_lo, msk_lo;
    int need, done;
};

__device__ __forceinline__ bool rank_less(uint64_t ah, uint32_t al, uint64_t bh, uint32_t bl) {
    return ah < bh || (ah == bh && al < bl);
}

__global__ void __launch_bounds__(SELECT_THREADS)
k_select(const Img* __restrict__ imgs, const Call* __restrict__ call) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ uint32_t hist[256];
    __shared__ SelState st;
    __shared__ int s_cnt;

    const Img& I = imgs[blockIdx.x];
    const int n = min(I.ctr[0], I.cand_cap);
    const int q = I.quota;
    const int tid = threadIdx.x;
    if (q <= 0 || n <= 0) {
        if (tid == 0) I.ctr[1] = 0;
        return;
    }
    const int m = min(n, q);
    int P = 1;
    while (P < m) P <<= 1;
    uint64_t* skey = reinterpret_cast<uint64_t*>(dyn);
    uint32_t* syx = reinterpret_cast<uint32_t*>(dyn + sizeof(uint64_t) * (size_t)P);

    if (tid == 0) {
        st.pre_hi = 0;
        st.msk_hi = 0;
        st.pre_lo = 0;
        st.msk_lo = 0;
        st.need = q;
        st.done = (n <= q);
        s_cnt = 0;
    }
    __syncthreads();

    for (int pass = 0; pass < 12 && !st.done; ++pass) {
        for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        const uint64_t pre_hi = st.pre_hi, msk_hi = st.msk_hi;
        const uint32_t pre_lo = st.pre_lo, msk_lo = st.msk_lo;
        const int shift_hi = 56 - 8 * pass, shift_lo = 24 - 8 * (pass - 8);
        for (int i = tid; i < n; i += blockDim.x) {
            const uint64_t hi = I.ckey[i];
            const uint32_t lo = ~I.cyx[i];
            if ((hi & msk_hi) == pre_hi && (lo & msk_lo) == pre_lo) {
                const uint32_t d = pass < 8 ? (uint32_t)(hi >> shift_hi) & 255u
                                            : (lo >> shift_lo) & 255u;
                atomicAdd(&hist[d], 1u);
            }
        }
        __syncthreads();
        if (tid == 0) {
            int need = st.need, cum = 0, d = 255;
            for (; d > 0; --d) {
                if (cum + (int)hist[d] >= need) break;
                cum += (int)hist[d];
            }
            need -= cum;
            if (pass < 8) {
                st.pre_hi |= (uint64_t)d << shift_hi;
                st.msk_hi |= 0xFFull << shift_hi;
            } else {
                st.pre_lo |= (uint32_t)d << shift_lo;
                st.msk_lo |= 0xFFu << shift_lo;
            }
            st.need = need;
            st.done = ((int)hist[d] == need);
        }
        __syncthreads();
    }

    // Gather: every candidate whose masked rank word is >= the fixed prefix.
    {
        const uint64_t pre_hi = st.pre_hi, msk_hi = st.msk_hi;
        const uint32_t pre_lo = st.pre_lo, msk_lo = st.msk_lo;
        for (int i = tid; i < n; i += blockDim.x) {
            const uint64_t hi = I.ckey[i];
            const uint32_t yx = I.cyx[i];
            const uint64_t mh = hi & msk_hi;
            const uint32_t ml = ~yx & msk_lo;
            if (mh > pre_hi || (mh == pre_hi && ml >= pre_lo)) {
                const int pos = atomicAdd(&s_cnt, 1);
                if (pos < P) {
                    skey[pos] = hi;
                    syx[pos] = yx;
                }
            }
        }
    }
    __syncthreads();
    const int got = min(s_cnt, m);
    for (int i = got + tid; i < P; i += blockDim.x) {
        skey[i] = 0ull;           // below every real candidate (keys never reach -2^63)
        syx[i] = 0xFFFFFFFFu;
    }
    __syncthreads();

    // Bitonic sort, descending by (key, ~yx).
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = tid; i < P; i += blockDim.x) {
                const int l = i ^ jj;
                if (l > i) {
                    const uint64_t ah = skey[i], bh = skey[l];
                    const uint32_t ay = syx[i], by = syx[l];
                    const bool a_less = rank_less(ah, ~ay, bh, ~by);
                    const bool desc = (i & k) == 0;
                    if (desc ? a_less : !a_less) {
                        skey[i] = bh;
                        skey[l] = ah;
                        syx[i] = by;
                        syx[l] = ay;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < got; i += blockDim.x) {
        I.kkey[i] = skey[i];
        I.kyx[i] = syx[i];
    }
    if (tid == 0) I.ctr[1] = got;
}

int select_smem_bytes(int max_quota) {
    int P = 1;
    while (P < max_quota) P <<= 1;
    return P * (int)(sizeof(uint64_t) + sizeof(uint32_t));
}

void launch_select(const Img* imgs, int n_img, const Call* call, int max_quota, void* stream) {
    if (n_img <= 0) return;
    const int smem = select_smem_bytes(max_quota > 0 ? max_quota : 1);
    k_select<<<n_img, SELECT_THREADS, smem, (cudaStream_t)stream>>>(imgs, call);
}

void set_select_smem_limit(int bytes) {
    cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace ofk
