// Tile-proposal network: forward, backward, Adam, checkpoints.
//
// The paper has no learned part; this network decides, per 32 x 32 tile of a
// pyramid level, whether the exact detector needs to run there.  Input: the
// tile with a 16-pixel halo (64 x 64 uint8, zero outside the image),
// normalised to (v - 128) / 64.  Layers (3 x 3 kernels, stride 2, padding 1,
// ReLU): 1 -> 8 channels (32 x 32), 8 -> 16 (16 x 16), 16 -> 16 (8 x 8);
// global average pool; linear 16 -> 1 logit.  Weights are stored and used as
// bf16 (rounded from fp32 master copies that Adam updates); every product is
// accumulated in fp32.  One block per tile; activations stay in shared
// memory.  Training uses a plain forward that saves activations to global
// memory for the backward pass; inference uses a register-blocked forward.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "of_internal.h"
#include "ofast.h"

namespace ofk {
void set_last_error(const std::string& msg);
}

namespace tn {

constexpr int S0 = 64, S1 = 32, S2 = 16, S3 = 8;  // spatial sizes
constexpr int C1 = 8, C2 = 16, C3 = 16;
// Flat parameter layout.
constexpr int W1 = 0, B1 = W1 + C1 * 9, W2 = B1 + C1, B2 = W2 + C2 * C1 * 9, W3 = B2 + C2,
              B3 = W3 + C3 * C2 * 9, WF = B3 + C3, BF = WF + C3, NP = BF + 1;
constexpr int A1 = C1 * S1 * S1, A2 = C2 * S2 * S2, A3 = C3 * S3 * S3;  // activation sizes
constexpr int SAVE = A1 + A2 + A3 + C3 + 1;  // per tile: a1, a2, a3, gap, logit
constexpr int THREADS = 256;
constexpr int SMEM_FWD = (S0 * S0 + A1 + A2 + A3 + NP + 32) * 4;

static_assert(NP == 3585, "parameter count");

}  // namespace tn

struct of_tcnn {
    float* master = nullptr;  // fp32 master weights [NP]
    __nv_bfloat16* w = nullptr;  // bf16 compute weights [NP]
    float* grad = nullptr;    // fp32 gradients [NP]
    float* m = nullptr;       // Adam moments
    float* v = nullptr;
    float* save = nullptr;    // saved activations [cap * SAVE]
    float* dz = nullptr;      // dLoss/dlogit [cap]
    float* loss = nullptr;    // [1]
    int cap = 0;
    int64_t step = 0;
    int device = 0;
};

namespace tn {

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// Source of one 64 x 64 input patch: either a dense tile array, or a
// proposal tile of a pyramid level read in place.
struct PatchSrc {
    const uint8_t* tiles;   // dense: n x 4096 bytes, or nullptr
    const ofk::Img* imgs;   // in place: image descriptors
    const int32_t* list;    // image index per job
    const int32_t* prefix;  // first tile of each job
    int n_list;
};

__device__ void load_patch(const PatchSrc& S, int t, float* in, int border) {
    if (S.tiles) {
        const uint8_t* p = S.tiles + (size_t)t * S0 * S0;
        for (int i = threadIdx.x; i < S0 * S0; i += blockDim.x) in[i] = ((float)p[i] - 128.f) * (1.f / 64.f);
        return;
    }
    int lo = 0, hi = S.n_list - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(S.prefix + mid) <= t) lo = mid; else hi = mid - 1;
    }
    const ofk::Img& I = S.imgs[__ldg(S.list + lo)];
    const int k = t - __ldg(S.prefix + lo);
    const int ptx = I.tiles_x * 4;
    const int x0 = I.tile_x0 + 32 * (k % ptx) - 16, y0 = border + 32 * (k / ptx) - 16;
    for (int i = threadIdx.x; i < S0 * S0; i += blockDim.x) {
        const int x = x0 + (i & 63), y = y0 + (i >> 6);
        // Pixels outside the image are 0 in the uint8 patch, i.e. -2 after normalisation.
        const float v = (x >= 0 && x < I.w && y >= 0 && y < I.h) ? (float)I.img[(size_t)y * I.pitch + x] : 0.f;
        in[i] = (v - 128.f) * (1.f / 64.f);
    }
}

// out[o][y][x] = relu(b[o] + sum_c sum_k w[o][c][k] in[c][2y+ky-1][2x+kx-1])
__device__ void conv_s2(const float* __restrict__ in, int C, int Sin, const float* __restrict__ w,
                        const float* __restrict__ b, int O, float* __restrict__ out) {
    const int Sout = Sin / 2;
    for (int i = threadIdx.x; i < O * Sout * Sout; i += blockDim.x) {
        const int o = i / (Sout * Sout), y = (i / Sout) % Sout, x = i % Sout;
        float acc = b[o];
        for (int c = 0; c < C; ++c) {
            const float* wc = w + (o * C + c) * 9;
            const float* ic = in + c * Sin * Sin;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int iy = 2 * y + ky - 1;
                if (iy < 0 || iy >= Sin) continue;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int ix = 2 * x + kx - 1;
                    if (ix < 0 || ix >= Sin) continue;
                    acc = fmaf(wc[ky * 3 + kx], ic[iy * Sin + ix], acc);
                }
            }
        }
        out[i] = relu(acc);
    }
}

// Forward pass of tiles [0, n); logits to `logits` (may be null); when `save`
// is set, activations to save[t * SAVE ...].
__global__ void __launch_bounds__(THREADS)
k_forward(PatchSrc src, int n, const __nv_bfloat16* __restrict__ wq, float* __restrict__ logits,
          float* __restrict__ save, int border) {
    extern __shared__ float sm[];
    float* in = sm;
    float* a1 = in + S0 * S0;
    float* a2 = a1 + A1;
    float* a3 = a2 + A2;
    float* w = a3 + A3;
    float* red = w + NP;
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __bfloat162float(wq[i]);
    __syncthreads();
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        load_patch(src, t, in, border);
        __syncthreads();
        conv_s2(in, 1, S0, w + W1, w + B1, C1, a1);
        __syncthreads();
        conv_s2(a1, C1, S1, w + W2, w + B2, C2, a2);
        __syncthreads();
        conv_s2(a2, C2, S2, w + W3, w + B3, C3, a3);
        __syncthreads();
        // Global average pool (one warp per 2 channels) and the linear head.
        if (threadIdx.x < 32 * 8) {
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            for (int c = warp; c < C3; c += 8) {
                float s = a3[c * 64 + lane] + a3[c * 64 + 32 + lane];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                if (lane == 0) red[c] = s * (1.f / 64.f);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float z = w[BF];
            for (int c = 0; c < C3; ++c) z = fmaf(w[WF + c], red[c], z);
            red[16] = z;
            if (logits) logits[t] = z;
        }
        __syncthreads();
        if (save) {
            float* sv = save + (size_t)t * SAVE;
            for (int i = threadIdx.x; i < A1; i += blockDim.x) sv[i] = a1[i];
            for (int i = threadIdx.x; i < A2; i += blockDim.x) sv[A1 + i] = a2[i];
            for (int i = threadIdx.x; i < A3; i += blockDim.x) sv[A1 + A2 + i] = a3[i];
            if (threadIdx.x <= C3) sv[A1 + A2 + A3 + threadIdx.x] = red[threadIdx.x];
        }
        __syncthreads();
    }
}

// Inference forward, register-blocked.  Activations live in zero-padded
// planes (no bounds tests); weights are transposed to [c][k][o] so one
// 16-byte broadcast load serves four output channels; a thread accumulates
// all channels of one output pixel (layers 1, 2) or four channels (layer 3).
// Same function as k_forward; products are summed over (c, ky, kx) in the
// same order.
constexpr int P0 = S0 + 2, P1 = S1 + 2, P2 = S2 + 2;
constexpr int FAST_SMEM = (P0 * P0 + C1 * P1 * P1 + C2 * P2 * P2 + A3 + NP + 32) * 4;

__global__ void __launch_bounds__(THREADS)
k_forward_fast(PatchSrc src, int n, const __nv_bfloat16* __restrict__ wq, float* __restrict__ logits, int border) {
    extern __shared__ __align__(16) float sm[];
    float* in = sm;                    // P0 x P0
    float* a1 = in + P0 * P0;          // C1 x P1 x P1
    float* a2 = a1 + C1 * P1 * P1;     // C2 x P2 x P2
    float* a3 = a2 + C2 * P2 * P2;     // C3 x 8 x 8
    float* w = a3 + A3;                // transposed weights + biases + head
    float* red = w + NP;
    const int tid = threadIdx.x;
    // Zero everything once: padding cells are never written afterwards.
    for (int i = tid; i < (int)(FAST_SMEM / 4); i += blockDim.x) sm[i] = 0.f;
    __syncthreads();
    // w1t[k][o], w2t[c][k][o], w3t[c][k][o] at the same offsets as W1, W2, W3.
    for (int i = tid; i < NP; i += blockDim.x) {
        float v = __bfloat162float(wq[i]);
        int dst = i;
        if (i < B1) {  // W1[o][0][k]
            const int o = i / 9, k = i % 9;
            dst = W1 + k * C1 + o;
        } else if (i >= W2 && i < B2) {
            const int j = i - W2, o = j / (C1 * 9), c = (j / 9) % C1, k = j % 9;
            dst = W2 + (c * 9 + k) * C2 + o;
        } else if (i >= W3 && i < B3) {
            const int j = i - W3, o = j / (C2 * 9), c = (j / 9) % C2, k = j % 9;
            dst = W3 + (c * 9 + k) * C3 + o;
        }
        w[dst] = v;
    }
    __syncthreads();
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        // Input patch into the interior of the padded plane.
        if (src.tiles) {
            const uint8_t* p = src.tiles + (size_t)t * S0 * S0;
            for (int i = tid; i < S0 * S0; i += blockDim.x)
                in[((i >> 6) + 1) * P0 + (i & 63) + 1] = ((float)p[i] - 128.f) * (1.f / 64.f);
        } else {
            int lo = 0, hi = src.n_list - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(src.prefix + mid) <= t) lo = mid; else hi = mid - 1;
            }
            const ofk::Img& I = src.imgs[__ldg(src.list + lo)];
            const int k = t - __ldg(src.prefix + lo);
            const int ptx = I.tiles_x * 4;
            const int x0 = I.tile_x0 + 32 * (k % ptx) - 16, y0 = border + 32 * (k / ptx) - 16;
            for (int i = tid; i < S0 * S0; i += blockDim.x) {
                const int x = x0 + (i & 63), y = y0 + (i >> 6);
                const float v = (x >= 0 && x < I.w && y >= 0 && y < I.h) ? (float)I.img[(size_t)y * I.pitch + x] : 0.f;
                in[((i >> 6) + 1) * P0 + (i & 63) + 1] = (v - 128.f) * (1.f / 64.f);
            }
        }
        __syncthreads();
        // Layer 1: 32 x 32 pixels, 4 per thread, 8 channels each.
        for (int px = tid; px < S1 * S1; px += blockDim.x) {
            const int y = px >> 5, x = px & 31;
            float acc[C1];
#pragma unroll
            for (int o = 0; o < C1; ++o) acc[o] = w[B1 + o];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float v = in[(2 * y + k / 3) * P0 + 2 * x + k % 3];
                const float4 wa = *reinterpret_cast<const float4*>(w + W1 + k * C1);
                const float4 wb = *reinterpret_cast<const float4*>(w + W1 + k * C1 + 4);
                acc[0] = fmaf(wa.x, v, acc[0]); acc[1] = fmaf(wa.y, v, acc[1]);
                acc[2] = fmaf(wa.z, v, acc[2]); acc[3] = fmaf(wa.w, v, acc[3]);
                acc[4] = fmaf(wb.x, v, acc[4]); acc[5] = fmaf(wb.y, v, acc[5]);
                acc[6] = fmaf(wb.z, v, acc[6]); acc[7] = fmaf(wb.w, v, acc[7]);
            }
#pragma unroll
            for (int o = 0; o < C1; ++o) a1[o * P1 * P1 + (y + 1) * P1 + x + 1] = relu(acc[o]);
        }
        __syncthreads();
        // Layer 2: 16 x 16 pixels, one per thread, 16 channels each.
        {
            const int y = tid >> 4, x = tid & 15;
            float acc[C2];
#pragma unroll
            for (int o = 0; o < C2; ++o) acc[o] = w[B2 + o];
            for (int c = 0; c < C1; ++c) {
                const float* ic = a1 + c * P1 * P1;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float v = ic[(2 * y + k / 3) * P1 + 2 * x + k % 3];
                    const float* wk = w + W2 + (c * 9 + k) * C2;
#pragma unroll
                    for (int o4 = 0; o4 < C2; o4 += 4) {
                        const float4 ww = *reinterpret_cast<const float4*>(wk + o4);
                        acc[o4] = fmaf(ww.x, v, acc[o4]);
                        acc[o4 + 1] = fmaf(ww.y, v, acc[o4 + 1]);
                        acc[o4 + 2] = fmaf(ww.z, v, acc[o4 + 2]);
                        acc[o4 + 3] = fmaf(ww.w, v, acc[o4 + 3]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < C2; ++o) a2[o * P2 * P2 + (y + 1) * P2 + x + 1] = relu(acc[o]);
        }
        __syncthreads();
        // Layer 3: 8 x 8 pixels x 4 channel groups.
        {
            const int pxl = tid & 63, g = tid >> 6;
            const int y = pxl >> 3, x = pxl & 7;
            float acc[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) acc[o] = w[B3 + 4 * g + o];
            for (int c = 0; c < C2; ++c) {
                const float* ic = a2 + c * P2 * P2;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const float v = ic[(2 * y + k / 3) * P2 + 2 * x + k % 3];
                    const float4 ww = *reinterpret_cast<const float4*>(w + W3 + (c * 9 + k) * C3 + 4 * g);
                    acc[0] = fmaf(ww.x, v, acc[0]); acc[1] = fmaf(ww.y, v, acc[1]);
                    acc[2] = fmaf(ww.z, v, acc[2]); acc[3] = fmaf(ww.w, v, acc[3]);
                }
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) a3[(4 * g + o) * 64 + pxl] = relu(acc[o]);
        }
        __syncthreads();
        {
            const int warp = tid >> 5, lane = tid & 31;
            for (int c = warp; c < C3; c += 8) {
                float sgap = a3[c * 64 + lane] + a3[c * 64 + 32 + lane];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sgap += __shfl_xor_sync(0xFFFFFFFFu, sgap, o);
                if (lane == 0) red[c] = sgap * (1.f / 64.f);
            }
        }
        __syncthreads();
        if (tid == 0) {
            float z = w[BF];
            for (int c = 0; c < C3; ++c) z = fmaf(w[WF + c], red[c], z);
            logits[t] = z;
        }
        __syncthreads();
    }
}

// Weighted BCE with logits: loss = mean_i w_i (softplus(z_i) - y_i z_i),
// w_i = pos_weight for y_i = 1; dz_i = w_i (sigmoid(z_i) - y_i) / n.
__global__ void k_bce(const float* __restrict__ save, const float* __restrict__ y, int n, float pos_weight,
                      float* __restrict__ dz, float* __restrict__ loss) {
    float acc = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float z = save[(size_t)i * SAVE + A1 + A2 + A3 + C3];
        const float wt = y[i] > 0.5f ? pos_weight : 1.f;
        const float sp = z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z));
        acc += wt * (sp - y[i] * z);
        const float sg = 1.f / (1.f + expf(-z));
        dz[i] = wt * (sg - y[i]) / (float)n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (float)n);
}

// Backward of one strided conv layer given dout (already multiplied by the
// ReLU derivative): accumulates dW, dB into gw, gb and writes din (without
// the input's ReLU derivative) when din is not null.
__device__ void conv_s2_back(const float* __restrict__ in, int C, int Sin, const float* __restrict__ w, int O,
                             const float* __restrict__ dout, float* __restrict__ gw, float* __restrict__ gb,
                             float* __restrict__ din) {
    const int Sout = Sin / 2;
    // dW[o][c][k] = sum_{y,x} dout[o][y][x] in[c][2y+ky-1][2x+kx-1]
    for (int i = threadIdx.x; i < O * C * 9; i += blockDim.x) {
        const int o = i / (C * 9), c = (i / 9) % C, k = i % 9, ky = k / 3, kx = k % 3;
        float acc = 0.f;
        for (int y = 0; y < Sout; ++y) {
            const int iy = 2 * y + ky - 1;
            if (iy < 0 || iy >= Sin) continue;
            for (int x = 0; x < Sout; ++x) {
                const int ix = 2 * x + kx - 1;
                if (ix < 0 || ix >= Sin) continue;
                acc = fmaf(dout[(o * Sout + y) * Sout + x], in[(c * Sin + iy) * Sin + ix], acc);
            }
        }
        gw[i] += acc;
    }
    for (int o = threadIdx.x; o < O; o += blockDim.x) {
        float acc = 0.f;
        for (int j = 0; j < Sout * Sout; ++j) acc += dout[o * Sout * Sout + j];
        gb[o] += acc;
    }
    if (!din) return;
    // din[c][iy][ix] = sum_{o,ky,kx} dout[o][y][x] w[o][c][ky][kx], iy = 2y+ky-1, ix = 2x+kx-1
    for (int i = threadIdx.x; i < C * Sin * Sin; i += blockDim.x) {
        const int c = i / (Sin * Sin), iy = (i / Sin) % Sin, ix = i % Sin;
        float acc = 0.f;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int ty = iy + 1 - ky;
            if (ty < 0 || (ty & 1) || (ty >> 1) >= Sout) continue;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int tx = ix + 1 - kx;
                if (tx < 0 || (tx & 1) || (tx >> 1) >= Sout) continue;
                for (int o = 0; o < O; ++o)
                    acc = fmaf(dout[(o * Sout + (ty >> 1)) * Sout + (tx >> 1)], w[(o * C + c) * 9 + ky * 3 + kx], acc);
            }
        }
        din[i] = acc;
    }
}

// Backward over tiles; per-block gradient sums in shared memory, added to
// `grad` once per block.
__global__ void __launch_bounds__(THREADS)
k_backward(const uint8_t* __restrict__ tiles, int n, const __nv_bfloat16* __restrict__ wq,
           const float* __restrict__ save, const float* __restrict__ dz, float* __restrict__ grad) {
    extern __shared__ float sm[];
    float* in = sm;                 // S0*S0
    float* d1 = in + S0 * S0;       // A1
    float* d2 = d1 + A1;            // A2
    float* d3 = d2 + A2;            // A3
    float* w = d3 + A3;             // NP
    float* g = w + NP;              // NP
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        w[i] = __bfloat162float(wq[i]);
        g[i] = 0.f;
    }
    __syncthreads();
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const float* sv = save + (size_t)t * SAVE;
        const float* a1 = sv;
        const float* a2 = sv + A1;
        const float* a3 = sv + A1 + A2;
        const float* gap = sv + A1 + A2 + A3;
        const float dl = dz[t];
        const uint8_t* p = tiles + (size_t)t * S0 * S0;
        for (int i = threadIdx.x; i < S0 * S0; i += blockDim.x) in[i] = ((float)p[i] - 128.f) * (1.f / 64.f);
        for (int c = threadIdx.x; c < C3; c += blockDim.x) g[WF + c] += dl * gap[c];
        if (threadIdx.x == 0) g[BF] += dl;
        // d3 = dgap / 64 * relu'(a3)
        for (int i = threadIdx.x; i < A3; i += blockDim.x) {
            const int c = i / 64;
            d3[i] = a3[i] > 0.f ? dl * w[WF + c] * (1.f / 64.f) : 0.f;
        }
        __syncthreads();
        conv_s2_back(a2, C2, S2, w + W3, C3, d3, g + W3, g + B3, d2);
        __syncthreads();
        for (int i = threadIdx.x; i < A2; i += blockDim.x) d2[i] = a2[i] > 0.f ? d2[i] : 0.f;
        __syncthreads();
        conv_s2_back(a1, C1, S1, w + W2, C2, d2, g + W2, g + B2, d1);
        __syncthreads();
        for (int i = threadIdx.x; i < A1; i += blockDim.x) d1[i] = a1[i] > 0.f ? d1[i] : 0.f;
        __syncthreads();
        conv_s2_back(in, 1, S0, w + W1, C1, d1, g + W1, g + B1, nullptr);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < NP; i += blockDim.x) atomicAdd(&grad[i], g[i]);
}

__global__ void k_adam(float* __restrict__ master, __nv_bfloat16* __restrict__ wq, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                       float wd, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / c1) / (sqrtf(vi / c2) + eps) + wd * master[i];
    const float w = master[i] - lr * upd;
    master[i] = w;
    wq[i] = __float2bfloat16_rn(w);
}

__global__ void k_round(const float* __restrict__ master, __nv_bfloat16* __restrict__ wq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) wq[i] = __float2bfloat16_rn(master[i]);
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ wq, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) out[i] = __bfloat162float(wq[i]);
}

uint32_t crc32(const uint8_t* p, size_t n) {
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; ++i) {
        c ^= p[i];
        for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
    }
    return ~c;
}

int fail(int code, const std::string& m) {
    ofk::set_last_error(m);
    return code;
}

int ensure_cap(of_tcnn* N, int n) {
    if (n <= N->cap) return OF_OK;
    if (N->save) cudaFree(N->save);
    if (N->dz) cudaFree(N->dz);
    N->save = nullptr;
    N->dz = nullptr;
    if (cudaMalloc(&N->save, sizeof(float) * SAVE * (size_t)n) != cudaSuccess ||
        cudaMalloc(&N->dz, sizeof(float) * (size_t)n) != cudaSuccess) {
        N->cap = 0;
        return fail(OF_ERR_CUDA, "tile-net workspace allocation failed");
    }
    N->cap = n;
    return OF_OK;
}

int grid_for(int n) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    return n < 2 * sms ? n : 2 * sms;
}

constexpr int SMEM_BWD = (S0 * S0 + A1 + A2 + A3 + 2 * NP) * 4;

// Proposal mask of one listed image per block (see of_detect_learned).
__global__ void k_propose(const ofk::Img* __restrict__ imgs, const int32_t* __restrict__ list,
                          const int32_t* __restrict__ prefix, const float* __restrict__ logits,
                          uint8_t* __restrict__ pos, uint8_t* __restrict__ mask, float threshold, float min_conf,
                          int dilate, int32_t* __restrict__ stats) {
    __shared__ float red[32];
    __shared__ int fallback, nprop;
    const int j = blockIdx.x;
    const ofk::Img& I = imgs[list[j]];
    const int base = prefix[j], n = prefix[j + 1] - base;
    const int ptx = 4 * I.tiles_x;
    float conf = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float p = 1.f / (1.f + expf(-logits[base + i]));
        conf += fabsf(2.f * p - 1.f);
        pos[base + i] = (p >= threshold) ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) conf += __shfl_xor_sync(0xFFFFFFFFu, conf, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = conf;
    if (threadIdx.x == 0) nprop = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        float c = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c += red[w];
        fallback = n > 0 && c / (float)n < min_conf;
    }
    __syncthreads();
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        uint8_t on = 1;
        if (!fallback) {
            const int px = i % ptx, py = i / ptx;
            on = pos[base + i];
            if (dilate && !on) {
                for (int dy = -1; dy <= 1 && !on; ++dy)
                    for (int dx = -1; dx <= 1 && !on; ++dx) {
                        const int qx = px + dx, qy = py + dy;
                        if (qx >= 0 && qx < ptx && qy >= 0 && qy < I.tiles_y) on = pos[base + qy * ptx + qx];
                    }
            }
        }
        mask[base + i] = on;
        cnt += on;
    }
    atomicAdd(&nprop, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&stats[0], n);
        atomicAdd(&stats[1], nprop);
        if (fallback) atomicAdd(&stats[2], 1);
    }
}

// Patches of every proposal tile of one image, tile-major.
__global__ void k_extract(const ofk::Img* __restrict__ imgs, int img, int border, uint8_t* __restrict__ dst, int n) {
    const ofk::Img& I = imgs[img];
    const int ptx = 4 * I.tiles_x;
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int x0 = I.tile_x0 + 32 * (t % ptx) - 16, y0 = border + 32 * (t / ptx) - 16;
        for (int i = threadIdx.x; i < S0 * S0; i += blockDim.x) {
            const int x = x0 + (i & 63), y = y0 + (i >> 6);
            dst[(size_t)t * S0 * S0 + i] =
                (x >= 0 && x < I.w && y >= 0 && y < I.h) ? I.img[(size_t)y * I.pitch + x] : (uint8_t)0;
        }
    }
}

}  // namespace tn

namespace ofk {
int launch_propose(const Img* imgs, const int32_t* list, const int32_t* prefix, int n_list, const float* logits,
                   uint8_t* pos, uint8_t* mask, float threshold, float min_conf, int dilate, int32_t* stats,
                   void* stream) {
    if (n_list <= 0) return OF_OK;
    tn::k_propose<<<n_list, 256, 0, (cudaStream_t)stream>>>(imgs, list, prefix, logits, pos, mask, threshold,
                                                            min_conf, dilate, stats);
    return cudaGetLastError() == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "proposal launch failed");
}

int launch_extract(const Img* imgs, int img, int border, uint8_t* dst, int n, void* stream) {
    if (n <= 0) return OF_OK;
    tn::k_extract<<<n < 1024 ? n : 1024, 256, 0, (cudaStream_t)stream>>>(imgs, img, border, dst, n);
    return cudaGetLastError() == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "extract launch failed");
}

// Forward over the proposal tiles of a batch (in place from the pyramid).
int tcnn_forward_tiles(of_tcnn* N, const Img* imgs, const int32_t* list, const int32_t* prefix, int n_list,
                       int n_tiles, int border, float* logits, void* stream) {
    if (n_tiles <= 0) return OF_OK;
    tn::PatchSrc src{nullptr, imgs, list, prefix, n_list};
    tn::k_forward_fast<<<tn::grid_for(n_tiles), tn::THREADS, tn::FAST_SMEM, (cudaStream_t)stream>>>(
        src, n_tiles, N->w, logits, border);
    return cudaGetLastError() == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "tile-net forward launch failed");
}
}  // namespace ofk

extern "C" {

of_tcnn* of_tcnn_create(uint64_t seed) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tn::k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, tn::SMEM_FWD);
        cudaFuncSetAttribute(tn::k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, tn::SMEM_BWD);
        cudaFuncSetAttribute(tn::k_forward_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, tn::FAST_SMEM);
        attr = true;
    }
    of_tcnn* N = new of_tcnn();
    cudaGetDevice(&N->device);
    const size_t b = sizeof(float) * tn::NP;
    if (cudaMalloc(&N->master, b) != cudaSuccess || cudaMalloc(&N->w, sizeof(__nv_bfloat16) * tn::NP) != cudaSuccess ||
        cudaMalloc(&N->grad, b) != cudaSuccess || cudaMalloc(&N->m, b) != cudaSuccess ||
        cudaMalloc(&N->v, b) != cudaSuccess || cudaMalloc(&N->loss, sizeof(float)) != cudaSuccess) {
        tn::fail(OF_ERR_CUDA, "tile-net allocation failed");
        of_tcnn_destroy(N);
        return nullptr;
    }
    // He-uniform initialisation from a 64-bit LCG (host), biases 0.
    std::vector<float> p(tn::NP, 0.f);
    uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto uni = [&]() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return (float)((s >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    };
    auto fill = [&](int off, int count, int fan_in) {
        const float a = std::sqrt(6.f / (float)fan_in);
        for (int i = 0; i < count; ++i) p[off + i] = a * uni();
    };
    fill(tn::W1, tn::C1 * 9, 9);
    fill(tn::W2, tn::C2 * tn::C1 * 9, tn::C1 * 9);
    fill(tn::W3, tn::C3 * tn::C2 * 9, tn::C2 * 9);
    fill(tn::WF, tn::C3, tn::C3);
    if (of_tcnn_set_params(N, p.data()) != OF_OK) {
        of_tcnn_destroy(N);
        return nullptr;
    }
    return N;
}

void of_tcnn_destroy(of_tcnn* N) {
    if (!N) return;
    for (void* q : {(void*)N->master, (void*)N->w, (void*)N->grad, (void*)N->m, (void*)N->v, (void*)N->save,
                    (void*)N->dz, (void*)N->loss})
        if (q) cudaFree(q);
    delete N;
}

int of_tcnn_num_params(void) { return tn::NP; }

int of_tcnn_set_params(of_tcnn* N, const float* host) {
    if (!N || !host) return tn::fail(OF_ERR_ARG, "null argument");
    const size_t b = sizeof(float) * tn::NP;
    if (cudaMemcpy(N->master, host, b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(N->m, 0, b) != cudaSuccess || cudaMemset(N->v, 0, b) != cudaSuccess ||
        cudaMemset(N->grad, 0, b) != cudaSuccess)
        return tn::fail(OF_ERR_CUDA, "tile-net upload failed");
    tn::k_round<<<(tn::NP + 255) / 256, 256>>>(N->master, N->w);
    N->step = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "tile-net rounding failed");
}

int of_tcnn_get_params(of_tcnn* N, int which, float* host) {
    if (!N || !host || which < 0 || which > 2) return tn::fail(OF_ERR_ARG, "bad arguments");
    const size_t b = sizeof(float) * tn::NP;
    cudaError_t e;
    if (which == 0) {
        e = cudaMemcpy(host, N->master, b, cudaMemcpyDeviceToHost);
    } else if (which == 2) {
        e = cudaMemcpy(host, N->grad, b, cudaMemcpyDeviceToHost);
    } else {
        float* tmp = nullptr;
        e = cudaMalloc(&tmp, b);
        if (e == cudaSuccess) {
            tn::k_bf16_to_f32<<<(tn::NP + 255) / 256, 256>>>(N->w, tmp);
            e = cudaMemcpy(host, tmp, b, cudaMemcpyDeviceToHost);
            cudaFree(tmp);
        }
    }
    return e == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "tile-net download failed");
}

int of_tcnn_forward(of_tcnn* N, const uint8_t* tiles, int n, float* logits, void* stream) {
    if (!N || !tiles || !logits || n < 0) return tn::fail(OF_ERR_ARG, "bad arguments");
    if (n == 0) return OF_OK;
    tn::PatchSrc src{tiles, nullptr, nullptr, nullptr, 0};
    tn::k_forward_fast<<<tn::grid_for(n), tn::THREADS, tn::FAST_SMEM, (cudaStream_t)stream>>>(src, n, N->w, logits,
                                                                                          0);
    return cudaGetLastError() == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "tile-net forward launch failed");
}

int of_tcnn_loss_grad(of_tcnn* N, const uint8_t* tiles, const float* labels, int n, float pos_weight,
                      float* loss_out, void* stream) {
    if (!N || !tiles || !labels || n < 1 || !(pos_weight > 0.f)) return tn::fail(OF_ERR_ARG, "bad arguments");
    int rc = tn::ensure_cap(N, n);
    if (rc != OF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(N->grad, 0, sizeof(float) * tn::NP, st);
    cudaMemsetAsync(N->loss, 0, sizeof(float), st);
    tn::PatchSrc src{tiles, nullptr, nullptr, nullptr, 0};
    tn::k_forward<<<tn::grid_for(n), tn::THREADS, tn::SMEM_FWD, st>>>(src, n, N->w, nullptr, N->save, 0);
    tn::k_bce<<<(n + 255) / 256, 256, 0, st>>>(N->save, labels, n, pos_weight, N->dz, N->loss);
    tn::k_backward<<<tn::grid_for(n), tn::THREADS, tn::SMEM_BWD, st>>>(tiles, n, N->w, N->save, N->dz, N->grad);
    if (cudaGetLastError() != cudaSuccess) return tn::fail(OF_ERR_CUDA, "tile-net training launch failed");
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, N->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return tn::fail(OF_ERR_CUDA, "tile-net loss readback failed");
    }
    return OF_OK;
}

int of_tcnn_adam(of_tcnn* N, float lr, float beta1, float beta2, float eps, float weight_decay, void* stream) {
    if (!N || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return tn::fail(OF_ERR_ARG, "bad Adam arguments");
    N->step += 1;
    const float c1 = 1.f - std::pow(beta1, (float)N->step), c2 = 1.f - std::pow(beta2, (float)N->step);
    tn::k_adam<<<(tn::NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(N->master, N->w, N->grad, N->m, N->v, lr,
                                                                        beta1, beta2, eps, weight_decay, c1, c2);
    return cudaGetLastError() == cudaSuccess ? OF_OK : tn::fail(OF_ERR_CUDA, "Adam launch failed");
}

// Checkpoint: "OFTC" | version u32 | n_params u32 | step i64 | master | m | v | crc32 of all before it.
int64_t of_tcnn_save(of_tcnn* N, uint8_t* buf, int64_t cap) {
    if (!N) return tn::fail(OF_ERR_ARG, "null net");
    const size_t body = 4 + 4 + 4 + 8 + 3 * sizeof(float) * tn::NP;
    const int64_t total = (int64_t)body + 4;
    if (!buf) return total;
    if (cap < total) return tn::fail(OF_ERR_ARG, "buffer too small");
    std::vector<float> a(tn::NP), m(tn::NP), v(tn::NP);
    if (cudaMemcpy(a.data(), N->master, sizeof(float) * tn::NP, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(m.data(), N->m, sizeof(float) * tn::NP, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(v.data(), N->v, sizeof(float) * tn::NP, cudaMemcpyDeviceToHost) != cudaSuccess)
        return tn::fail(OF_ERR_CUDA, "download failed");
    uint8_t* p = buf;
    std::memcpy(p, "OFTC", 4);
    const uint32_t ver = 1, np = tn::NP;
    std::memcpy(p + 4, &ver, 4);
    std::memcpy(p + 8, &np, 4);
    std::memcpy(p + 12, &N->step, 8);
    std::memcpy(p + 20, a.data(), sizeof(float) * tn::NP);
    std::memcpy(p + 20 + sizeof(float) * tn::NP, m.data(), sizeof(float) * tn::NP);
    std::memcpy(p + 20 + 2 * sizeof(float) * tn::NP, v.data(), sizeof(float) * tn::NP);
    const uint32_t crc = tn::crc32(buf, body);
    std::memcpy(p + body, &crc, 4);
    return total;
}

int of_tcnn_load(of_tcnn* N, const uint8_t* buf, int64_t n) {
    if (!N || !buf) return tn::fail(OF_ERR_ARG, "null argument");
    const size_t body = 4 + 4 + 4 + 8 + 3 * sizeof(float) * tn::NP;
    if (n != (int64_t)body + 4) return tn::fail(OF_ERR_ARG, "checkpoint size mismatch");
    uint32_t ver, np, crc;
    std::memcpy(&ver, buf + 4, 4);
    std::memcpy(&np, buf + 8, 4);
    std::memcpy(&crc, buf + body, 4);
    if (std::memcmp(buf, "OFTC", 4) != 0 || ver != 1 || np != (uint32_t)tn::NP)
        return tn::fail(OF_ERR_ARG, "not a version-1 tile-net checkpoint");
    if (tn::crc32(buf, body) != crc) return tn::fail(OF_ERR_ARG, "checkpoint CRC mismatch");
    const int rc = of_tcnn_set_params(N, reinterpret_cast<const float*>(buf + 20));
    if (rc != OF_OK) return rc;
    std::memcpy(&N->step, buf + 12, 8);
    if (cudaMemcpy(N->m, buf + 20 + sizeof(float) * tn::NP, sizeof(float) * tn::NP, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(N->v, buf + 20 + 2 * sizeof(float) * tn::NP, sizeof(float) * tn::NP, cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return tn::fail(OF_ERR_CUDA, "upload failed");
    return OF_OK;
}

}  // extern "C"
