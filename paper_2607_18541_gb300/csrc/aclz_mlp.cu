// Learned per-block thresholds: block features and a small FP32 MLP
// (24 -> 64 -> 64 -> K, ReLU, softmax cross-entropy, Adam), trained and run
// with these kernels.
//
// The paper's lever (Sec. IV-B, IV-C) is a fixed vector of minimum match
// lengths by distance class; its cause (Sec. IV-C) is that short copies
// from distant positions cost more in offset bits than the literals they
// replace, and give the decoding warp too little work.  The network picks, per block, one of K candidate vectors from
// statistics of the block, so blocks can take a different point on that
// trade-off.  Sizes are tiny (6.5k parameters), so the contractions run on
// CUDA cores; tiles of 32 samples keep activations in shared memory and
// per-tile gradient partials are reduced in a fixed order (deterministic).
#include <cmath>

#include "aclz_device.cuh"
#include "aclz_internal.h"

using namespace aclz;

namespace {

constexpr int kIn = 24, kHid = 64, kMaxK = 16, kTile = 32, kMlpThreads = 256;

__host__ __device__ constexpr uint32_t param_count(uint32_t K) {
    return kIn * kHid + kHid + kHid * kHid + kHid + kHid * K + K;
}

struct Off {
    uint32_t W1, b1, W2, b2, W3, b3, P;
};
__host__ __device__ inline Off offsets(uint32_t K) {
    Off o;
    o.W1 = 0;
    o.b1 = o.W1 + kIn * kHid;
    o.W2 = o.b1 + kHid;
    o.b2 = o.W2 + kHid * kHid;
    o.W3 = o.b2 + kHid;
    o.b3 = o.W3 + kHid * K;
    o.P = o.b3 + K;
    return o;
}

// One tile of 32 samples: forward; with TRAIN, softmax cross-entropy and
// the backward pass, writing this tile's gradient partial (P floats) and
// summed loss to part[tile * (P + 1)].
template <bool TRAIN>
__global__ void __launch_bounds__(kMlpThreads) k_mlp_tile(const float *__restrict__ p, uint32_t K,
                                                          const float *__restrict__ x,
                                                          const int32_t *__restrict__ y, uint32_t B,
                                                          float *__restrict__ logits,
                                                          float *__restrict__ part) {
    __shared__ float xs[kTile][kIn];
    __shared__ float h1[kTile][kHid], h2[kTile][kHid];
    __shared__ float dz[kTile][kMaxK], d2[kTile][kHid], d1[kTile][kHid];
    __shared__ float ls[kTile];
    const Off o = offsets(K);
    const int tid = threadIdx.x;
    const uint32_t s0 = blockIdx.x * kTile;
    const uint32_t ns = min((uint32_t)kTile, B - s0);
    for (int i = tid; i < kTile * kIn; i += kMlpThreads) {
        const int s = i / kIn, c = i % kIn;
        xs[s][c] = (uint32_t)s < ns ? x[(size_t)(s0 + s) * kIn + c] : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kTile * kHid; i += kMlpThreads) {
        const int s = i / kHid, j = i % kHid;
        float a = p[o.b1 + j];
        for (int c = 0; c < kIn; c++) a += xs[s][c] * p[o.W1 + c * kHid + j];
        h1[s][j] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kTile * kHid; i += kMlpThreads) {
        const int s = i / kHid, j = i % kHid;
        float a = p[o.b2 + j];
        for (int c = 0; c < kHid; c++) a += h1[s][c] * p[o.W2 + c * kHid + j];
        h2[s][j] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kTile * (int)K; i += kMlpThreads) {
        const int s = i / K, k = i % K;
        float a = p[o.b3 + k];
        for (int c = 0; c < kHid; c++) a += h2[s][c] * p[o.W3 + c * K + k];
        dz[s][k] = a;
        if (!TRAIN && (uint32_t)s < ns) logits[(size_t)(s0 + s) * K + k] = a;
    }
    __syncthreads();
    if (!TRAIN) return;
    if (tid < kTile) {
        const int s = tid;
        if ((uint32_t)s < ns) {
            float m = dz[s][0];
            for (uint32_t k = 1; k < K; k++) m = fmaxf(m, dz[s][k]);
            float den = 0.f;
            for (uint32_t k = 0; k < K; k++) den += expf(dz[s][k] - m);
            int yy = y[s0 + s];
            yy = yy < 0 ? 0 : (yy >= (int)K ? (int)K - 1 : yy);  // labels are checked on the host
            ls[s] = -(dz[s][yy] - m - logf(den));
            for (uint32_t k = 0; k < K; k++)
                dz[s][k] = (expf(dz[s][k] - m) / den - (k == (uint32_t)yy ? 1.f : 0.f)) / (float)B;
        } else {
            ls[s] = 0.f;
            for (uint32_t k = 0; k < K; k++) dz[s][k] = 0.f;
        }
    }
    __syncthreads();
    float *g = part + (size_t)blockIdx.x * (o.P + 1);
    for (int i = tid; i < kHid * (int)K; i += kMlpThreads) {
        const int j = i / K, k = i % K;
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += h2[s][j] * dz[s][k];
        g[o.W3 + j * K + k] = a;
    }
    for (int k = tid; k < (int)K; k += kMlpThreads) {
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += dz[s][k];
        g[o.b3 + k] = a;
    }
    for (int i = tid; i < kTile * kHid; i += kMlpThreads) {
        const int s = i / kHid, j = i % kHid;
        float a = 0.f;
        for (uint32_t k = 0; k < K; k++) a += dz[s][k] * p[o.W3 + j * K + k];
        d2[s][j] = h2[s][j] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kHid * kHid; i += kMlpThreads) {
        const int c = i / kHid, j = i % kHid;
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += h1[s][c] * d2[s][j];
        g[o.W2 + c * kHid + j] = a;
    }
    for (int j = tid; j < kHid; j += kMlpThreads) {
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += d2[s][j];
        g[o.b2 + j] = a;
    }
    for (int i = tid; i < kTile * kHid; i += kMlpThreads) {
        const int s = i / kHid, c = i % kHid;
        float a = 0.f;
        for (int j = 0; j < kHid; j++) a += d2[s][j] * p[o.W2 + c * kHid + j];
        d1[s][c] = h1[s][c] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kIn * kHid; i += kMlpThreads) {
        const int c = i / kHid, j = i % kHid;
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += xs[s][c] * d1[s][j];
        g[o.W1 + c * kHid + j] = a;
    }
    for (int j = tid; j < kHid; j += kMlpThreads) {
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += d1[s][j];
        g[o.b1 + j] = a;
    }
    if (tid == 0) {
        float a = 0.f;
        for (int s = 0; s < kTile; s++) a += ls[s];
        g[o.P] = a;
    }
}

// grad[p] = sum over tiles in order; loss = (sum of tile losses) / B
__global__ void k_mlp_reduce(const float *__restrict__ part, uint32_t tiles, uint32_t P, uint32_t B,
                             float *__restrict__ grad, float *__restrict__ loss) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= P; i += gridDim.x * blockDim.x) {
        float a = 0.f;
        for (uint32_t t = 0; t < tiles; t++) a += part[(size_t)t * (P + 1) + i];
        if (i < P) grad[i] = a;
        else if (loss) *loss = a / (float)B;
    }
}

// Adam with bias correction; c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
__global__ void k_adam(float *p, float *m, float *v, const float *__restrict__ g, uint32_t P, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Byte statistics of one LZ block per CTA:
// order-0 entropy, distinct values, repeats of the previous byte, repeat
// rates of 4- and 8-grams by linear counting over a 65536-bit map, and
// byte-class fractions.
constexpr int kFeatThreads = 256;
__global__ void __launch_bounds__(kFeatThreads) k_block_features(const uint8_t *__restrict__ x, uint64_t n,
                                                                 uint32_t bs, float *__restrict__ feat) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t bm4[2048], bm8[2048];
    __shared__ uint32_t cnt[8];
    __shared__ float red[kFeatThreads / 32];
    const int tid = threadIdx.x;
    const uint64_t b0 = (uint64_t)blockIdx.x * bs;
    const uint32_t m = (uint32_t)((uint64_t)bs < n - b0 ? (uint64_t)bs : n - b0);
    for (int i = tid; i < 256; i += kFeatThreads) hist[i] = 0;
    for (int i = tid; i < 2048; i += kFeatThreads) bm4[i] = bm8[i] = 0;
    if (tid < 8) cnt[tid] = 0;
    __syncthreads();
    const uint8_t *s = x + b0;
    uint32_t rep = 0, dig = 0, low = 0, up = 0, pun = 0;
    for (uint32_t i = tid; i < m; i += kFeatThreads) {
        const uint32_t c = s[i];
        atomicAdd(&hist[c], 1u);
        if (i > 0 && s[i - 1] == c) rep++;
        dig += (c >= 0x30 && c <= 0x39);
        low += (c >= 0x61 && c <= 0x7A);
        up += (c >= 0x41 && c <= 0x5A);
        pun += ((c >= 0x20 && c <= 0x2F) || (c >= 0x3A && c <= 0x40) || (c >= 0x5B && c <= 0x60) ||
                (c >= 0x7B && c <= 0x7E));
        if (i + 4 <= m) {
            unsigned long long k = 0;
            for (int j = 0; j < 4; j++) k |= (unsigned long long)s[i + j] << (8 * j);
            const uint32_t hsh = (uint32_t)((k * 0x9E3779B97F4A7C15ULL) >> 48);
            atomicOr(&bm4[hsh >> 5], 1u << (hsh & 31));
            if (i + 8 <= m) {
                for (int j = 4; j < 8; j++) k |= (unsigned long long)s[i + j] << (8 * j);
                const uint32_t h8 = (uint32_t)((k * 0x9E3779B97F4A7C15ULL) >> 48);
                atomicOr(&bm8[h8 >> 5], 1u << (h8 & 31));
            }
        }
    }
    atomicAdd(&cnt[0], rep);
    atomicAdd(&cnt[1], dig);
    atomicAdd(&cnt[2], low);
    atomicAdd(&cnt[3], up);
    atomicAdd(&cnt[4], pun);
    __syncthreads();
    // entropy and distinct values
    float e = 0.f;
    uint32_t distinct = 0;
    for (int i = tid; i < 256; i += kFeatThreads) {
        const uint32_t h = hist[i];
        if (h) {
            const float pr = (float)h / (float)m;
            e -= pr * log2f(pr);
            distinct++;
        }
    }
    uint32_t set4 = 0, set8 = 0;
    for (int i = tid; i < 2048; i += kFeatThreads) {
        set4 += __popc(bm4[i]);
        set8 += __popc(bm8[i]);
    }
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
        set4 += __shfl_xor_sync(0xffffffffu, set4, o);
        set8 += __shfl_xor_sync(0xffffffffu, set8, o);
    }
    if ((tid & 31) == 0) {
        red[tid >> 5] = e;
        atomicAdd(&cnt[5], distinct);
        atomicAdd(&cnt[6], set4);
        atomicAdd(&cnt[7], set8);
    }
    __syncthreads();
    if (tid == 0) {
        float et = 0.f;
        for (int w = 0; w < kFeatThreads / 32; w++) et += red[w];
        float *f = feat + (size_t)blockIdx.x * 10;
        f[0] = et / 8.f;
        f[1] = (float)cnt[5] / 256.f;
        f[2] = m > 1 ? (float)cnt[0] / (float)m : 0.f;
        const uint32_t sets[2] = {cnt[6], cnt[7]};
        const uint32_t ks[2] = {4, 8};
        for (int q = 0; q < 2; q++) {
            float r = 0.f;
            if (m >= ks[q]) {
                const float pos = (float)(m - ks[q] + 1);
                const uint32_t z = 65536u - sets[q];
                float est = -65536.f * logf((float)(z ? z : 1u) / 65536.f);
                est = fminf(est, pos);
                r = 1.f - est / pos;
            }
            f[3 + q] = r;
        }
        f[5] = (float)cnt[1] / (float)m;
        f[6] = (float)cnt[2] / (float)m;
        f[7] = (float)cnt[3] / (float)m;
        f[8] = (float)cnt[4] / (float)m;
        f[9] = 1.f - (f[5] + f[6] + f[7] + f[8]);
    }
}

int last_error() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return ACLZ_E_CUDA;
    }
    return ACLZ_OK;
}

}  // namespace

extern "C" uint32_t aclz_mlp_param_count(uint32_t K) { return param_count(K); }

extern "C" uint64_t aclz_mlp_scratch_bytes(uint32_t K, uint32_t batch) {
    const uint64_t tiles = (batch + kTile - 1) / kTile;
    return tiles * (param_count(K) + 1) * sizeof(float);
}

extern "C" int aclz_mlp_forward(const float *d_params, uint32_t K, const float *d_x, uint32_t batch,
                                float *d_logits, void *stream) {
    if (!d_params || K < 2 || K > kMaxK || (batch && (!d_x || !d_logits))) return ACLZ_E_INVAL;
    if (!batch) return ACLZ_OK;
    const unsigned tiles = (batch + kTile - 1) / kTile;
    k_mlp_tile<false><<<tiles, kMlpThreads, 0, (cudaStream_t)stream>>>(d_params, K, d_x, nullptr, batch, d_logits,
                                                                        nullptr);
    return last_error();
}

extern "C" int aclz_mlp_grad(const float *d_params, uint32_t K, const float *d_x, const int32_t *d_y,
                             uint32_t batch, float *d_grad, float *d_loss, void *d_scratch, uint64_t scratch_bytes,
                             void *stream) {
    if (!d_params || K < 2 || K > kMaxK || !batch || !d_x || !d_y || !d_grad || !d_scratch) return ACLZ_E_INVAL;
    if (scratch_bytes < aclz_mlp_scratch_bytes(K, batch)) return ACLZ_E_CAPACITY;
    const unsigned tiles = (batch + kTile - 1) / kTile;
    cudaStream_t st = (cudaStream_t)stream;
    float *part = (float *)d_scratch;
    k_mlp_tile<true><<<tiles, kMlpThreads, 0, st>>>(d_params, K, d_x, d_y, batch, nullptr, part);
    k_mlp_reduce<<<(param_count(K) + 256) / 256, 256, 0, st>>>(part, tiles, param_count(K), batch, d_grad, d_loss);
    return last_error();
}

extern "C" int aclz_mlp_adam(float *d_params, float *d_m, float *d_v, const float *d_grad, uint32_t K,
                             uint32_t step, float lr, void *stream) {
    if (!d_params || !d_m || !d_v || !d_grad || K < 2 || K > kMaxK || step == 0) return ACLZ_E_INVAL;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)step)));
    const uint32_t P = param_count(K);
    k_adam<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_params, d_m, d_v, d_grad, P, lr, (float)b1,
                                                              (float)b2, 1e-8f, c1, c2);
    return last_error();
}

extern "C" int aclz_block_features(const void *d_x, uint64_t n, uint32_t block_size, float *d_feat, void *stream) {
    if ((n && (!d_x || !d_feat)) || block_size == 0) return ACLZ_E_INVAL;
    const uint64_t nb = (n + block_size - 1) / block_size;
    if (!nb) return ACLZ_OK;
    if (nb > 0x7fffffffULL) return ACLZ_E_UNSUPPORTED;
    k_block_features<<<(unsigned)nb, kFeatThreads, 0, (cudaStream_t)stream>>>((const uint8_t *)d_x, n, block_size,
                                                                            d_feat);
    return last_error();
}
