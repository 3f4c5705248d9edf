// Top-N per level: keep the n_l best NMS survivors of each (frame, level)
// image in rank order -- Harris key descending, then y ascending, then x
// ascending (Harris "screens" the FAST points, Sec. 1 and Sec. 3.2).
//
// One block per image.  Each candidate has a unique 96-bit rank word
//   R = (key ^ 2^63) << 32 | ~((y << 16) | x),
// larger R = better rank.  The candidates above the n_l-th largest R are
// found in one of two ways:
//   - coarse pass: a 4096-bin histogram of a code of the key that is
//     monotone in the key (sign, bit length and the next 5 bits of |key|)
//     locates the bin b holding the n_l-th largest key; every candidate with
//     code >= b is gathered (when they fit in shared memory) and sorted,
//     and the first n_l are kept;
//   - otherwise an MSB-first radix select over 8-bit digits of R (one
//     shared-memory histogram per pass) fixes, digit by digit, the prefix of
//     the n_l-th largest R, stopping as soon as every candidate that shares
//     the fixed prefix is needed, and those candidates are gathered.
// The gathered candidates are bitonic-sorted by R, descending.  The largest
// images hold tens of thousands of candidates, so every scan over them keeps
// SEL_UNROLL loads in flight per thread (the scans are latency-bound, not
// bandwidth-bound); the coarse passes load two keys per 16-byte load and read
// the positions of the gathered candidates only.
#include <cuda_runtime.h>

#include <mutex>

#include "of_internal.h"

namespace ofk {

constexpr int SEL_UNROLL = 4;   // candidates loaded per thread before use
constexpr int SEL_BINS = 4096;  // coarse-pass histogram bins
constexpr int SEL_MAX_DYN = 192 * 1024;

struct SelState {
    uint64_t pre_hi, msk_hi;
    uint32_t pre_lo, msk_lo;
    int need, done;
    int coarse, code_b, n_take;
};

__device__ __forceinline__ bool rank_less(uint64_t ah, uint32_t al, uint64_t bh, uint32_t bl) {
    return ah < bh || (ah == bh && al < bl);
}

// f(x) for 0 <= x < 2^63: 0 for x = 0, else 32 * bitlength(x) + the 5 bits
// after the leading one -- non-decreasing in x, at most 2047.
__device__ __forceinline__ uint32_t mag_code(uint64_t x) {
    if (x == 0ull) return 0u;
    const int L = 64 - __clzll((long long)x);
    return 32u * (uint32_t)L + (uint32_t)((x << (64 - L)) >> 58 & 31ull);
}

// Code of the order-preserving key u = key ^ 2^63, non-decreasing in key:
// keys >= 0 map to 2048 + f(key), keys < 0 to 2047 - f(-key - 1).
__device__ __forceinline__ uint32_t key_code(uint64_t u) {
    return (u >> 63) ? 2048u + mag_code(u & 0x7FFFFFFFFFFFFFFFull) : 2047u - mag_code(u ^ 0x7FFFFFFFFFFFFFFFull);
}

__global__ void __launch_bounds__(SELECT_THREADS)
k_select(const Img* __restrict__ imgs, const Call* __restrict__ call, int sort_cap) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ uint32_t hist[SEL_BINS];
    __shared__ uint32_t wsum[SELECT_THREADS / 32];
    __shared__ SelState st;
    __shared__ int s_cnt;

    const Img& I = imgs[blockIdx.x];
    const int n = min(I.ctr[0], I.cand_cap);
    const int q = I.quota;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (q <= 0 || n <= 0) {
        if (tid == 0) I.ctr[1] = 0;
        return;
    }
    const int m = min(n, q);
    uint64_t* skey = reinterpret_cast<uint64_t*>(dyn);
    uint32_t* syx = reinterpret_cast<uint32_t*>(dyn + sizeof(uint64_t) * (size_t)sort_cap);

    if (tid == 0) {
        st.pre_hi = 0;
        st.msk_hi = 0;
        st.pre_lo = 0;
        st.msk_lo = 0;
        st.need = q;
        st.done = (n <= q);
        st.coarse = 0;
        st.code_b = 0;
        st.n_take = m;
        s_cnt = 0;
    }
    for (int i = tid; i < SEL_BINS; i += SELECT_THREADS) hist[i] = 0u;
    __syncthreads();

    if (n > q) {
        // Coarse pass: histogram of the key code, two keys per 16-byte load
        // (the candidate arrays start on 256-byte boundaries).
        const ulonglong2* ck2 = reinterpret_cast<const ulonglong2*>(I.ckey);
        const int n2 = n >> 1;
        for (int i0 = tid; i0 < n2; i0 += SEL_UNROLL * SELECT_THREADS) {
            ulonglong2 v[SEL_UNROLL];
#pragma unroll
            for (int k = 0; k < SEL_UNROLL; ++k) {
                const int i = i0 + k * SELECT_THREADS;
                v[k] = i < n2 ? __ldg(ck2 + i) : make_ulonglong2(0ull, 0ull);
            }
#pragma unroll
            for (int k = 0; k < SEL_UNROLL; ++k)
                if (i0 + k * SELECT_THREADS < n2) {
                    atomicAdd(&hist[key_code(v[k].x)], 1u);
                    atomicAdd(&hist[key_code(v[k].y)], 1u);
                }
        }
        if ((n & 1) && tid == 0) atomicAdd(&hist[key_code(__ldg(I.ckey + n - 1))], 1u);
        __syncthreads();
        // Suffix sums: thread t owns bins [8t, 8t + 8); higher bins = better keys.
        constexpr int PER = SEL_BINS / SELECT_THREADS;
        const int b0 = tid * PER;
        int own = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) own += (int)hist[b0 + j];
        int v = own;  // sum over this warp's lanes >= lane
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_down_sync(0xFFFFFFFFu, v, off);
            if (lane + off < 32) v += t;
        }
        if (lane == 0) wsum[warp] = (uint32_t)v;
        __syncthreads();
        int above = v - own;
        for (int w = warp + 1; w < SELECT_THREADS / 32; ++w) above += (int)wsum[w];
        if (above < q && above + own >= q) {  // exactly one thread: the n_l-th best key is in its bins
            int cum = above;
            for (int j = PER - 1; j >= 0; --j) {
                const int h = (int)hist[b0 + j];
                if (cum + h >= q) {
                    st.code_b = b0 + j;
                    st.n_take = cum + h;
                    st.coarse = (cum + h <= sort_cap);
                    break;
                }
                cum += h;
            }
        }
        __syncthreads();
    }

    if (!st.coarse) {
        for (int pass = 0; pass < 12 && !st.done; ++pass) {
            for (int i = tid; i < 256; i += SELECT_THREADS) hist[i] = 0u;
            __syncthreads();
            const uint64_t pre_hi = st.pre_hi, msk_hi = st.msk_hi;
            const uint32_t pre_lo = st.pre_lo, msk_lo = st.msk_lo;
            const int shift_hi = 56 - 8 * pass, shift_lo = 24 - 8 * (pass - 8);
            const bool need_lo = pass >= 8;  // block-uniform
            for (int i0 = tid; i0 < n; i0 += SEL_UNROLL * SELECT_THREADS) {
                uint64_t hi[SEL_UNROLL];
                uint32_t lo[SEL_UNROLL];
#pragma unroll
                for (int k = 0; k < SEL_UNROLL; ++k) {
                    const int i = i0 + k * SELECT_THREADS;
                    hi[k] = i < n ? __ldg(I.ckey + i) : 0ull;
                    lo[k] = need_lo && i < n ? ~__ldg(I.cyx + i) : 0u;
                }
#pragma unroll
                for (int k = 0; k < SEL_UNROLL; ++k) {
                    if (i0 + k * SELECT_THREADS < n && (hi[k] & msk_hi) == pre_hi && (lo[k] & msk_lo) == pre_lo) {
                        const uint32_t d = pass < 8 ? (uint32_t)(hi[k] >> shift_hi) & 255u
                                                    : (lo[k] >> shift_lo) & 255u;
                        atomicAdd(&hist[d], 1u);
                    }
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
    }

    // Gather: code >= b (coarse), else every candidate whose masked rank word
    // is >= the fixed prefix.
    const bool coarse = st.coarse;  // block-uniform
    const int n_take = coarse ? st.n_take : m;
    {
        const uint64_t pre_hi = st.pre_hi, msk_hi = st.msk_hi;
        const uint32_t pre_lo = st.pre_lo, msk_lo = st.msk_lo;
        const uint32_t code_b = (uint32_t)st.code_b;
        if (coarse) {
            // Two keys per 16-byte load; positions only for the candidates taken.
            const ulonglong2* ck2 = reinterpret_cast<const ulonglong2*>(I.ckey);
            const int n2 = (n + 1) >> 1;
            for (int i0 = tid; i0 < n2; i0 += SEL_UNROLL * SELECT_THREADS) {
                ulonglong2 v[SEL_UNROLL];
#pragma unroll
                for (int k = 0; k < SEL_UNROLL; ++k) {
                    const int i = i0 + k * SELECT_THREADS;
                    if (i < n2) {
                        if (2 * i + 1 < n) v[k] = __ldg(ck2 + i);
                        else v[k] = make_ulonglong2(__ldg(I.ckey + 2 * i), 0ull);
                    } else {
                        v[k] = make_ulonglong2(0ull, 0ull);
                    }
                }
#pragma unroll
                for (int k = 0; k < SEL_UNROLL; ++k) {
                    const int i = i0 + k * SELECT_THREADS;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t key = h ? v[k].y : v[k].x;
                        if (i < n2 && 2 * i + h < n && key_code(key) >= code_b) {
                            const int pos = atomicAdd(&s_cnt, 1);
                            if (pos < sort_cap) {
                                skey[pos] = key;
                                syx[pos] = __ldg(I.cyx + 2 * i + h);
                            }
                        }
                    }
                }
            }
        } else
        for (int i0 = tid; i0 < n; i0 += SEL_UNROLL * SELECT_THREADS) {
            uint64_t hi[SEL_UNROLL];
            uint32_t yx[SEL_UNROLL];
#pragma unroll
            for (int k = 0; k < SEL_UNROLL; ++k) {
                const int i = i0 + k * SELECT_THREADS;
                hi[k] = i < n ? __ldg(I.ckey + i) : 0ull;
                yx[k] = i < n ? __ldg(I.cyx + i) : 0u;
            }
#pragma unroll
            for (int k = 0; k < SEL_UNROLL; ++k) {
                bool take;
                if (coarse) {
                    take = key_code(hi[k]) >= code_b;
                } else {
                    const uint64_t mh = hi[k] & msk_hi;
                    const uint32_t ml = ~yx[k] & msk_lo;
                    take = mh > pre_hi || (mh == pre_hi && ml >= pre_lo);
                }
                if (i0 + k * SELECT_THREADS < n && take) {
                    const int pos = atomicAdd(&s_cnt, 1);
                    if (pos < sort_cap) {
                        skey[pos] = hi[k];
                        syx[pos] = yx[k];
                    }
                }
            }
        }
    }
    __syncthreads();
    const int got = min(min(s_cnt, n_take), sort_cap);
    int P = 1;
    while (P < got) P <<= 1;
    for (int i = got + tid; i < P; i += SELECT_THREADS) {
        skey[i] = 0ull;           // below every real candidate (keys never reach -2^63)
        syx[i] = 0xFFFFFFFFu;
    }
    __syncthreads();

    // Bitonic sort, descending by (key, ~yx); one thread per compared pair.
    for (int k = 2; k <= P; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int p = tid; p < (P >> 1); p += SELECT_THREADS) {
                const int i = ((p & ~(jj - 1)) << 1) | (p & (jj - 1));
                const int l = i | jj;
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
            __syncthreads();
        }
    }
    const int out = min(got, m);
    for (int i = tid; i < out; i += SELECT_THREADS) {
        I.kkey[i] = skey[i];
        I.kyx[i] = syx[i];
    }
    if (tid == 0) I.ctr[1] = out;
}

// Sort-buffer entries: room for twice the largest quota (the coarse pass's
// boundary bin), else the quota rounded up to a power of two.
static int select_sort_cap(int max_quota) {
    int P = 1;
    while (P < max_quota) P <<= 1;
    return 2 * P * (int)(sizeof(uint64_t) + sizeof(uint32_t)) <= SEL_MAX_DYN ? 2 * P : P;
}

int select_smem_bytes(int max_quota) {
    return select_sort_cap(max_quota) * (int)(sizeof(uint64_t) + sizeof(uint32_t));
}

void launch_select(const Img* imgs, int n_img, const Call* call, int max_quota, void* stream) {
    if (n_img <= 0) return;
    const int mq = max_quota > 0 ? max_quota : 1;
    k_select<<<n_img, SELECT_THREADS, select_smem_bytes(mq), (cudaStream_t)stream>>>(imgs, call,
                                                                                      select_sort_cap(mq));
}

// The limit is a per-device attribute of the kernel shared by every handle,
// server slot and allocation-free call, so it only ever grows: a later caller
// with a smaller quota must not lower it under an earlier one.
void set_select_smem_limit(int bytes) {
    static std::mutex mu;
    static int limit[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && bytes <= limit[dev]) return;
    if (cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
        dev >= 0 && dev < 64)
        limit[dev] = bytes;
}

}  // namespace ofk
