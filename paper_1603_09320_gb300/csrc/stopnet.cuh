// stopnet.cuh -- the learned early-stop network shared by the search kernel
// (inference) and the training kernels.  The paper has no learned part; this
// is an addition beside the plain method.
//
// Network: x in R^6 -> (x - mu) / sigma -> relu(W1 . + b1) [64] ->
//          relu(W2 . + b2) [64] -> w3 . + b3 (a logit).  Weights are fp16
// values, arithmetic is fp32.  Parameter order of the fp16 vector
// (4,673 values): W1 (64 x 6, row-major out x in) | b1 | W2 (64 x 64) | b2 |
// w3 | b3.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hnswgb {

constexpr int kStopIn = 6;
constexpr int kStopH = 64;
constexpr int kStopParams = kStopIn * kStopH + kStopH + kStopH * kStopH + kStopH + kStopH + 1;  // 4673
constexpr int kOffW1 = 0, kOffB1 = 384, kOffW2 = 448, kOffB2 = 4544, kOffW3 = 4608, kOffB3 = 4672;

// Inference layout on the device: the input normalisation folded into the
// first layer (w1[j][i] = W1[j][i] / sigma[i], b1[j] - sum_i w1[j][i] mu[i],
// computed in double and rounded to fp32), the other small tensors widened to
// fp32 (exact), W2 kept in fp16 as pairs (W2[l][u], W2[l+32][u]) so that lane
// l of a warp reads one 4-byte word per input u.
struct StopDev {
    float w1[kStopH * kStopIn];
    float b1[kStopH];
    float b2[kStopH];
    float w3[kStopH];
    float b3;
    float pad[3];
    __half2 w2p[kStopH * 32];
};
static_assert(sizeof(StopDev) % 16 == 0, "StopDev is copied in 16-byte words");

// Loads of the network's weights: read-only global loads (GLOBAL) or plain
// shared-memory loads.
template <bool GLOBAL>
__device__ __forceinline__ float ldw(const float* p) {
    return GLOBAL ? __ldg(p) : *p;
}
template <bool GLOBAL>
__device__ __forceinline__ __half2 ldw(const __half2* p) {
    return GLOBAL ? __ldg(p) : *p;
}

// Logit of the network for features f (identical in every lane), computed by
// one warp from the network m (in global memory when GLOBAL, else the
// block's shared-memory copy): lane l owns hidden units l and l + 32.  The
// first hidden layer is exchanged through a 64-float scratch `hs` in shared
// memory and read back with 16-byte broadcast loads.
template <bool GLOBAL>
__device__ __forceinline__ float stop_logit(const StopDev* __restrict__ m, const float (&f)[kStopIn],
                                            float* hs, int lane) {
    float ha = ldw<GLOBAL>(m->b1 + lane), hb = ldw<GLOBAL>(m->b1 + lane + 32);
#pragma unroll
    for (int i = 0; i < kStopIn; ++i) {
        ha = fmaf(ldw<GLOBAL>(m->w1 + lane * kStopIn + i), f[i], ha);
        hb = fmaf(ldw<GLOBAL>(m->w1 + (lane + 32) * kStopIn + i), f[i], hb);
    }
    __syncwarp();
    hs[lane] = fmaxf(ha, 0.0f);
    hs[lane + 32] = fmaxf(hb, 0.0f);
    __syncwarp();
    // two accumulators per output (even and odd inputs) halve the FMA chains
    float za = ldw<GLOBAL>(m->b2 + lane), zb = ldw<GLOBAL>(m->b2 + lane + 32), za1 = 0.0f, zb1 = 0.0f;
    const float4* h4 = reinterpret_cast<const float4*>(hs);
#pragma unroll 4
    for (int u4 = 0; u4 < kStopH / 4; ++u4) {
        const float4 h = h4[u4];
        const float2 w0 = __half22float2(ldw<GLOBAL>(m->w2p + (u4 * 4 + 0) * 32 + lane));
        const float2 w1 = __half22float2(ldw<GLOBAL>(m->w2p + (u4 * 4 + 1) * 32 + lane));
        const float2 w2 = __half22float2(ldw<GLOBAL>(m->w2p + (u4 * 4 + 2) * 32 + lane));
        const float2 w3 = __half22float2(ldw<GLOBAL>(m->w2p + (u4 * 4 + 3) * 32 + lane));
        za = fmaf(w0.x, h.x, za);
        zb = fmaf(w0.y, h.x, zb);
        za1 = fmaf(w1.x, h.y, za1);
        zb1 = fmaf(w1.y, h.y, zb1);
        za = fmaf(w2.x, h.z, za);
        zb = fmaf(w2.y, h.z, zb);
        za1 = fmaf(w3.x, h.w, za1);
        zb1 = fmaf(w3.y, h.w, zb1);
    }
    za += za1;
    zb += zb1;
    float o = ldw<GLOBAL>(m->w3 + lane) * fmaxf(za, 0.0f) + ldw<GLOBAL>(m->w3 + lane + 32) * fmaxf(zb, 0.0f);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
    return o + ldw<GLOBAL>(&m->b3);
}

}  // namespace hnswgb
