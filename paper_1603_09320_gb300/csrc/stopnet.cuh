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

// Inference layout on the device: the small tensors widened to fp32 (exact),
// W2 kept in fp16 as pairs (W2[l][u], W2[l+32][u]) so that lane l of a warp
// reads one 4-byte word per input u.
struct StopDev {
    float mu[kStopIn];
    float isig[kStopIn];
    float w1[kStopH * kStopIn];
    float b1[kStopH];
    float b2[kStopH];
    float w3[kStopH];
    float b3;
    float pad[3];
    __half2 w2p[kStopH * 32];
};
static_assert(sizeof(StopDev) % 16 == 0, "StopDev is copied in 16-byte words");

// Logit of the network for features f (identical in every lane), computed by
// one warp from the block's shared-memory copy m of the network: lane l owns
// hidden units l and l + 32.  The first hidden layer is exchanged through a
// 64-float scratch `hs` in shared memory and read back with 16-byte
// broadcast loads.
__device__ __forceinline__ float stop_logit(const StopDev* __restrict__ m, const float (&f)[kStopIn],
                                            float* hs, int lane) {
    float xn[kStopIn];
#pragma unroll
    for (int i = 0; i < kStopIn; ++i) xn[i] = (f[i] - m->mu[i]) * m->isig[i];
    float ha = m->b1[lane], hb = m->b1[lane + 32];
#pragma unroll
    for (int i = 0; i < kStopIn; ++i) {
        ha = fmaf(m->w1[lane * kStopIn + i], xn[i], ha);
        hb = fmaf(m->w1[(lane + 32) * kStopIn + i], xn[i], hb);
    }
    __syncwarp();
    hs[lane] = fmaxf(ha, 0.0f);
    hs[lane + 32] = fmaxf(hb, 0.0f);
    __syncwarp();
    float za = m->b2[lane], zb = m->b2[lane + 32];
    const float4* h4 = reinterpret_cast<const float4*>(hs);
#pragma unroll 4
    for (int u4 = 0; u4 < kStopH / 4; ++u4) {
        const float4 h = h4[u4];
        const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 wf = __half22float2(m->w2p[(u4 * 4 + j) * 32 + lane]);
            za = fmaf(wf.x, hv[j], za);
            zb = fmaf(wf.y, hv[j], zb);
        }
    }
    float o = m->w3[lane] * fmaxf(za, 0.0f) + m->w3[lane + 32] * fmaxf(zb, 0.0f);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
    return o + m->b3;
}

}  // namespace hnswgb
