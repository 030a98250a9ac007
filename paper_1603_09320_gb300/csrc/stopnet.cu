// stopnet.cu -- training of the learned early-stop network on the GPU and
// its upload into an index (hnsw_stop_grad, hnsw_stop_train,
// hnsw_set_stop_model, hnsw_clear_stop_model).  The paper has no counterpart.
//
// Training is mini-batch gradient descent on the mean binary cross-entropy
// of sigmoid(logit) against the 0/1 labels, with Adam (fp32 master weights,
// fp16 working weights: the forward and backward passes use the fp16 values,
// as inference does).  One block runs the forward and backward pass of 128
// samples with all activations in shared memory and adds its parameter
// gradient into a global fp32 buffer; an optimiser kernel then updates the
// weights.  Samples are visited in a different affine order each epoch.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.hpp"
#include "index.cuh"
#include "stopnet.cuh"

namespace hnswgb {
namespace {

constexpr int kTB = 128;       // samples per block
constexpr int kThreads = 256;
constexpr int kLd = kStopH + 1;  // padded row of the activation tiles

struct TrainSmem {
    float w1[kStopH * kStopIn], b1[kStopH], w2[kStopH * kStopH], w2t[kStopH * kStopH], b2[kStopH], w3[kStopH], b3;
    float x[kTB * kStopIn], y[kTB], dz[kTB];
    float h1[kTB * kLd];  // relu(a1), later d(loss)/d(a1)
    float a2[kTB * kLd];  // a2, later d(loss)/d(a2)
    float mu[kStopIn], isig[kStopIn];
    float loss;
};

__device__ __forceinline__ int sample_index(int64_t i, int64_t n, uint64_t a, uint64_t c) {
    return int((a * uint64_t(i) + c) % uint64_t(n));
}

// Forward + backward of samples [base, base + kTB) of the epoch order
// (clipped to n); adds scale * gradient into grad and scale * loss into loss.
__global__ void __launch_bounds__(kThreads) stop_fwd_bwd(const float* __restrict__ X, const float* __restrict__ Y,
                                                         int64_t n, uint64_t pa, uint64_t pc, int64_t base0,
                                                         const float* __restrict__ norm,
                                                         const __half* __restrict__ w, float* __restrict__ grad,
                                                         float* __restrict__ loss, float scale) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(sm_raw);
    const int t = threadIdx.x;
    const int64_t base = base0 + int64_t(blockIdx.x) * kTB;
    const int nb = int(base >= n ? 0 : (n - base < kTB ? n - base : kTB));
    if (nb == 0) return;
    for (int i = t; i < kStopH * kStopIn; i += kThreads) S.w1[i] = __half2float(w[kOffW1 + i]);
    for (int i = t; i < kStopH * kStopH; i += kThreads) {
        const float v = __half2float(w[kOffW2 + i]);
        S.w2[i] = v;
        S.w2t[(i % kStopH) * kStopH + i / kStopH] = v;
    }
    for (int i = t; i < kStopH; i += kThreads) {
        S.b1[i] = __half2float(w[kOffB1 + i]);
        S.b2[i] = __half2float(w[kOffB2 + i]);
        S.w3[i] = __half2float(w[kOffW3 + i]);
    }
    if (t == 0) {
        S.b3 = __half2float(w[kOffB3]);
        S.loss = 0.0f;
    }
    if (t < kStopIn) {
        S.mu[t] = norm[t];
        S.isig[t] = 1.0f / norm[kStopIn + t];
    }
    __syncthreads();
    for (int i = t; i < kTB * kStopIn; i += kThreads) {
        const int b = i / kStopIn, f = i % kStopIn;
        S.x[i] = b < nb ? (X[int64_t(sample_index(base + b, n, pa, pc)) * kStopIn + f] - S.mu[f]) * S.isig[f] : 0.0f;
    }
    for (int b = t; b < kTB; b += kThreads) S.y[b] = b < nb ? Y[sample_index(base + b, n, pa, pc)] : 0.0f;
    __syncthreads();
    // h1 = relu(W1 x + b1)
    for (int i = t; i < kTB * kStopH; i += kThreads) {
        const int b = i / kStopH, o = i % kStopH;
        float a = S.b1[o];
#pragma unroll
        for (int f = 0; f < kStopIn; ++f) a = fmaf(S.w1[o * kStopIn + f], S.x[b * kStopIn + f], a);
        S.h1[b * kLd + o] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    // a2 = W2 h1 + b2
    for (int i = t; i < kTB * kStopH; i += kThreads) {
        const int b = i / kStopH, o = i % kStopH;
        float a = S.b2[o];
        for (int u = 0; u < kStopH; ++u) a = fmaf(S.w2t[u * kStopH + o], S.h1[b * kLd + u], a);
        S.a2[b * kLd + o] = a;
    }
    __syncthreads();
    // logit, loss, d loss / d logit
    if (t < kTB) {
        float z = S.b3;
        for (int o = 0; o < kStopH; ++o) z = fmaf(S.w3[o], fmaxf(S.a2[t * kLd + o], 0.0f), z);
        float dz = 0.0f, l = 0.0f;
        if (t < nb) {
            const float y = S.y[t];
            l = fmaxf(z, 0.0f) - z * y + log1pf(expf(-fabsf(z)));
            dz = (1.0f / (1.0f + expf(-z)) - y) * scale;
        }
        S.dz[t] = dz;
        for (int s = 16; s > 0; s >>= 1) l += __shfl_xor_sync(0xffffffffu, l, s);
        if ((t & 31) == 0) atomicAdd(&S.loss, l);
    }
    __syncthreads();
    // w3, b3 gradients; then a2 <- d loss / d a2
    if (t < kStopH) {
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g = fmaf(S.dz[b], fmaxf(S.a2[b * kLd + t], 0.0f), g);
        atomicAdd(&grad[kOffW3 + t], g);
    } else if (t == kStopH) {
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g += S.dz[b];
        atomicAdd(&grad[kOffB3], g);
    }
    __syncthreads();
    for (int i = t; i < kTB * kStopH; i += kThreads) {
        const int b = i / kStopH, o = i % kStopH;
        const float a = S.a2[b * kLd + o];
        S.a2[b * kLd + o] = a > 0.0f ? S.dz[b] * S.w3[o] : 0.0f;
    }
    __syncthreads();
    // W2, b2 gradients: sum over samples of d a2 (outer) h1
    for (int i = t; i < kStopH * kStopH; i += kThreads) {
        const int o = i / kStopH, u = i % kStopH;
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g = fmaf(S.a2[b * kLd + o], S.h1[b * kLd + u], g);
        atomicAdd(&grad[kOffW2 + i], g);
    }
    if (t < kStopH) {
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g += S.a2[b * kLd + t];
        atomicAdd(&grad[kOffB2 + t], g);
    }
    __syncthreads();
    // h1 <- d loss / d a1 = (W2^T d a2) masked by a1 > 0
    for (int i = t; i < kTB * kStopH; i += kThreads) {
        const int b = i / kStopH, u = i % kStopH;
        const float h = S.h1[b * kLd + u];
        float g = 0.0f;
        if (h > 0.0f)
            for (int o = 0; o < kStopH; ++o) g = fmaf(S.a2[b * kLd + o], S.w2[o * kStopH + u], g);
        S.h1[b * kLd + u] = g;
    }
    __syncthreads();
    // W1, b1 gradients
    for (int i = t; i < kStopH * kStopIn; i += kThreads) {
        const int o = i / kStopIn, f = i % kStopIn;
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g = fmaf(S.h1[b * kLd + o], S.x[b * kStopIn + f], g);
        atomicAdd(&grad[kOffW1 + i], g);
    }
    if (t < kStopH) {
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g += S.h1[b * kLd + t];
        atomicAdd(&grad[kOffB1 + t], g);
    }
    if (t == 0) atomicAdd(loss, S.loss * scale);
}

// Adam step on the fp32 master weights; writes the fp16 working copy and
// clears the gradient.
__global__ void stop_adam(float* __restrict__ master, __half* __restrict__ w16, float* __restrict__ grad,
                          float* __restrict__ m1, float* __restrict__ m2, float lr, float beta1, float beta2,
                          float eps, float wd, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kStopParams; i += gridDim.x * blockDim.x) {
        const float g = grad[i] + wd * master[i];
        const float a = beta1 * m1[i] + (1.0f - beta1) * g;
        const float b = beta2 * m2[i] + (1.0f - beta2) * g * g;
        m1[i] = a;
        m2[i] = b;
        const float p = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        master[i] = p;
        w16[i] = __float2half_rn(p);
        grad[i] = 0.0f;
    }
}

// Feature means and standard deviations (one block; sums in fp64).
__global__ void stop_norm(const float* __restrict__ X, int64_t n, float* __restrict__ norm) {
    __shared__ double s1[kStopIn][32], s2[kStopIn][32];
    double a[kStopIn] = {}, b[kStopIn] = {};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        for (int f = 0; f < kStopIn; ++f) {
            const double v = X[i * kStopIn + f];
            a[f] += v;
            b[f] += v * v;
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int f = 0; f < kStopIn; ++f) {
        for (int s = 16; s > 0; s >>= 1) {
            a[f] += __shfl_xor_sync(0xffffffffu, a[f], s);
            b[f] += __shfl_xor_sync(0xffffffffu, b[f], s);
        }
        if (lane == 0) {
            s1[f][wid] = a[f];
            s2[f][wid] = b[f];
        }
    }
    __syncthreads();
    if (threadIdx.x < kStopIn) {
        double sa = 0, sb = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            sa += s1[threadIdx.x][w];
            sb += s2[threadIdx.x][w];
        }
        const double mean = sa / double(n);
        const double var = sb / double(n) - mean * mean;
        norm[threadIdx.x] = float(mean);
        norm[kStopIn + threadIdx.x] = float(sqrt(var > 1e-12 ? var : 1e-12));
    }
}

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

hnsw_status cuda_err(cudaError_t e, const char* what) {
    return fail(HNSW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

bool bad_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return !(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
}

size_t smem_bytes() { return sizeof(TrainSmem); }

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

hnsw_status set_smem() {
    return raise_smem_limit(reinterpret_cast<const void*>(stop_fwd_bwd), smem_bytes(), "stop network");
}

}  // namespace
}  // namespace hnswgb

using namespace hnswgb;

extern "C" hnsw_status hnsw_stop_grad(const float* x, const float* y, int64_t n, const float* norm,
                                      const uint16_t* w_fp16, float* grad_out, float* loss_out, void* stream) {
    if (!x || !y || !norm || !w_fp16 || !grad_out || n < 1) return fail(HNSW_EINVAL, "hnsw_stop_grad: bad argument");
    if (bad_device_ptr(x) || bad_device_ptr(y)) return fail(HNSW_EINVAL, "hnsw_stop_grad: x and y must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hnsw_status st = set_smem();
    if (st != HNSW_OK) return st;
    DevBuf buf;
    // sections start on 256-byte boundaries: [fp16 weights][fp32 grad | loss | norm]
    const size_t off_g = round256(size_t(kStopParams) * 2);
    const size_t bytes = off_g + round256((kStopParams + 1 + 2 * kStopIn) * 4);
    cudaError_t e = cudaMalloc(&buf.p, bytes);
    if (e != cudaSuccess) return fail(HNSW_ENOMEM, "hnsw_stop_grad: device buffer");
    __half* dw = static_cast<__half*>(buf.p);
    float* dg = reinterpret_cast<float*>(static_cast<char*>(buf.p) + off_g);
    float* dl = dg + kStopParams;
    float* dn = dl + 1;
    if ((e = cudaMemcpyAsync(dw, w_fp16, kStopParams * 2, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dn, norm, 2 * kStopIn * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(dg, 0, (kStopParams + 1) * 4, s)) != cudaSuccess)
        return cuda_err(e, "hnsw_stop_grad: copy");
    const unsigned blocks = unsigned((n + kTB - 1) / kTB);
    stop_fwd_bwd<<<blocks, kThreads, smem_bytes(), s>>>(x, y, n, 1, 0, 0, dn, dw, dg, dl, 1.0f / float(n));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "hnsw_stop_grad: launch");
    if ((e = cudaMemcpyAsync(grad_out, dg, kStopParams * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_err(e, "hnsw_stop_grad: copy back");
    float l = 0;
    if ((e = cudaMemcpyAsync(&l, dl, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_err(e, "hnsw_stop_grad: sync");
    if (loss_out) *loss_out = l;
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_stop_train(const float* x, const float* y, int64_t n, const hnsw_stop_train_params* p,
                                       const uint16_t* w_init, float* norm_out, uint16_t* w_out,
                                       float* loss_per_epoch, void* stream) {
    if (!x || !y || !p || !w_init || !norm_out || !w_out || n < 1)
        return fail(HNSW_EINVAL, "hnsw_stop_train: bad argument");
    if (p->epochs < 1 || p->batch < kTB || p->batch % kTB != 0 || !(p->lr > 0))
        return fail(HNSW_EINVAL, "hnsw_stop_train: epochs >= 1, batch a multiple of 128, lr > 0");
    if (bad_device_ptr(x) || bad_device_ptr(y)) return fail(HNSW_EINVAL, "hnsw_stop_train: x and y must be device memory");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hnsw_status st = set_smem();
    if (st != HNSW_OK) return st;
    DevBuf buf;
    // sections on 256-byte boundaries: [fp16 weights][master][grad][m1][m2][norm][loss per epoch]
    const size_t sw = round256(size_t(kStopParams) * 2), sf = round256(size_t(kStopParams) * 4);
    const size_t bytes = sw + 4 * sf + 256 + round256(size_t(p->epochs) * 4);
    cudaError_t e = cudaMalloc(&buf.p, bytes);
    if (e != cudaSuccess) return fail(HNSW_ENOMEM, "hnsw_stop_train: device buffer");
    char* c = static_cast<char*>(buf.p);
    __half* dw = reinterpret_cast<__half*>(c);
    float* master = reinterpret_cast<float*>(c + sw);
    float* grad = reinterpret_cast<float*>(c + sw + sf);
    float* m1 = reinterpret_cast<float*>(c + sw + 2 * sf);
    float* m2 = reinterpret_cast<float*>(c + sw + 3 * sf);
    float* dn = reinterpret_cast<float*>(c + sw + 4 * sf);          // 12 floats
    float* dloss = reinterpret_cast<float*>(c + sw + 4 * sf + 256);  // epochs floats
    std::vector<float> mw(kStopParams);
    for (int i = 0; i < kStopParams; ++i) {
        __half_raw r;
        r.x = w_init[i];
        mw[i] = __half2float(__half(r));
    }
    if ((e = cudaMemcpyAsync(dw, w_init, kStopParams * 2, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(master, mw.data(), kStopParams * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(grad, 0, 3 * sf, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(dloss, 0, size_t(p->epochs) * 4, s)) != cudaSuccess)
        return cuda_err(e, "hnsw_stop_train: copy");
    stop_norm<<<1, 256, 0, s>>>(x, n, dn);
    const float b1 = p->beta1 > 0 ? p->beta1 : 0.9f, b2 = p->beta2 > 0 ? p->beta2 : 0.999f;
    const float eps = p->eps > 0 ? p->eps : 1e-8f;
    uint64_t rng = p->seed ^ 0x5eed5eedull;
    int step = 0;
    const int64_t steps_per_epoch = (n + p->batch - 1) / p->batch;
    for (int ep = 0; ep < p->epochs; ++ep) {
        // a new affine visiting order of the samples: i -> (a i + c) mod n
        uint64_t a = 1 + splitmix64(rng) % uint64_t(n);
        while (gcd64(a, uint64_t(n)) != 1) a = 1 + (a % uint64_t(n));
        const uint64_t cc = splitmix64(rng) % uint64_t(n);
        for (int64_t k = 0; k < steps_per_epoch; ++k) {
            const int64_t base = k * p->batch;
            const int64_t nb = n - base < p->batch ? n - base : p->batch;
            const unsigned blocks = unsigned((nb + kTB - 1) / kTB);
            stop_fwd_bwd<<<blocks, kThreads, smem_bytes(), s>>>(x, y, n, a, cc, base, dn, dw, grad, dloss + ep,
                                                                1.0f / float(nb));
            ++step;
            const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
            stop_adam<<<19, 256, 0, s>>>(master, dw, grad, m1, m2, p->lr, b1, b2, eps, p->weight_decay, c1, c2);
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "hnsw_stop_train: launch");
    if ((e = cudaMemcpyAsync(w_out, dw, kStopParams * 2, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(norm_out, dn, 2 * kStopIn * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_err(e, "hnsw_stop_train: copy back");
    std::vector<float> ls(p->epochs);
    if ((e = cudaMemcpyAsync(ls.data(), dloss, size_t(p->epochs) * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_err(e, "hnsw_stop_train: sync");
    if (loss_per_epoch)
        for (int i = 0; i < p->epochs; ++i) loss_per_epoch[i] = ls[i] / float(steps_per_epoch);
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_set_stop_model(hnsw_index* ix, const float* norm, const uint16_t* w_fp16) {
    if (!ix || !norm || !w_fp16) return fail(HNSW_EINVAL, "hnsw_set_stop_model: null argument");
    StopDev h{};
    auto f16 = [&](int i) {
        __half_raw r;
        r.x = w_fp16[i];
        return __half(r);
    };
    for (int i = 0; i < kStopIn; ++i)
        if (!(norm[kStopIn + i] > 0)) return fail(HNSW_EINVAL, "hnsw_set_stop_model: sigma must be > 0");
    // (x - mu) / sigma folded into the first layer
    for (int j = 0; j < kStopH; ++j) {
        double b = double(__half2float(f16(kOffB1 + j)));
        for (int i = 0; i < kStopIn; ++i) {
            const double w = double(__half2float(f16(kOffW1 + j * kStopIn + i))) / double(norm[kStopIn + i]);
            h.w1[j * kStopIn + i] = float(w);
            b -= w * double(norm[i]);
        }
        h.b1[j] = float(b);
    }
    for (int i = 0; i < kStopH; ++i) {
        h.b2[i] = __half2float(f16(kOffB2 + i));
        h.w3[i] = __half2float(f16(kOffW3 + i));
    }
    h.b3 = __half2float(f16(kOffB3));
    for (int u = 0; u < kStopH; ++u)
        for (int l = 0; l < 32; ++l) h.w2p[u * 32 + l] = __halves2half2(f16(kOffW2 + l * kStopH + u), f16(kOffW2 + (l + 32) * kStopH + u));
    if (!ix->d_stop) {
        cudaError_t e = cudaMalloc(&ix->d_stop, sizeof(StopDev));
        if (e != cudaSuccess) {
            ix->d_stop = nullptr;
            return fail(HNSW_ENOMEM, "hnsw_set_stop_model: device buffer");
        }
    }
    cudaError_t e = cudaMemcpy(ix->d_stop, &h, sizeof(StopDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(e, "hnsw_set_stop_model: copy");
    return HNSW_OK;
}

extern "C" hnsw_status hnsw_clear_stop_model(hnsw_index* ix) {
    if (!ix) return fail(HNSW_EINVAL, "hnsw_clear_stop_model: null index");
    if (ix->d_stop) {
        cudaDeviceSynchronize();
        cudaFree(ix->d_stop);
        ix->d_stop = nullptr;
    }
    return HNSW_OK;
}
