// Learned position index over the Hilbert-sorted keys of a layer's objects:
// the device-side model shared by the training kernels, the error-bound pass
// and the render kernel's candidate lookup.
//
// position(k) ~ j*P + c_j + a_j * (k - kb_j) + P * mlp(t, e_j)
//   j      piece of k (the last piece whose first key kb_j <= k; pieces are
//          P consecutive sorted keys), found through a radix table on the
//          top 16 key bits,
//   a, c   least-squares line of the piece,
//   t      (k - kb_j) / (kb_{j+1} - kb_j), e_j a 4-vector embedding of the
//          piece, mlp a 5 -> H -> H -> 1 ReLU network with bf16 weights and
//          fp32 accumulation, trained on the device on the residual; a piece
//          adds the MLP term only if that narrows its own error bound.
// Every stored key's true position lies within eps_j of its prediction
// (measured over all keys with this same code); a lookup searches that
// window, confirms the bracket, and falls back to a full binary search.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace hv {

constexpr int kLearnIn = 5;       // t and a 4-vector piece embedding
constexpr int kLearnH = 16;       // hidden width of the residual MLP
constexpr int kRadixBits = 16;    // radix table over the top 16 of 62 key bits

struct LModel {
    const uint64_t* keys;     // sorted keys, n
    uint64_t n;
    const uint64_t* kb;       // first key of each piece, n_seg
    const float* pa;          // slope, positions per key unit
    const float* pc;          // intercept within the piece
    const float* pinv;        // 1 / (kb_{j+1} - kb_j) (0 for the last piece)
    const uint32_t* eps;      // per-piece max position error (ceil)
    const uint32_t* rt;       // radix table, (1 << kRadixBits) + 2 entries
    const __nv_bfloat16* emb; // n_seg x 4
    const __nv_bfloat16* w;   // W1 [H x 5], b1 [H], W2 [H x H], b2 [H], w3 [H], b3
    const uint8_t* use_mlp;   // per piece: 1 if the MLP residual narrows its bound
    uint32_t n_seg;
    uint32_t P;
    int hidden;               // 0 = linear pieces only, else kLearnH
};

constexpr int kLearnNW = kLearnH * kLearnIn + kLearnH + kLearnH * kLearnH + kLearnH + kLearnH + 1;

// Last piece whose first key is <= k (0 when k precedes every piece).
__device__ __forceinline__ uint32_t learn_piece(const LModel& m, uint64_t k) {
    uint64_t t = k >> (62 - kRadixBits);
    if (t > (1u << kRadixBits)) t = 1u << kRadixBits;
    uint32_t lo = __ldg(m.rt + t), hi = __ldg(m.rt + t + 1);
    // answer in [lo - 1, hi - 1]
    int64_t a = (int64_t)lo - 1, b = (int64_t)hi - 1;
    if (a < 0) a = 0;
    if (b < a) b = a;
    while (a < b) {
        int64_t mid = (a + b + 1) >> 1;
        if (__ldg(m.kb + mid) <= k) a = mid; else b = mid - 1;
    }
    return (uint32_t)a;
}

// MLP residual in units of P (fp32 accumulation over bf16 weights).
__device__ __forceinline__ float learn_mlp(const LModel& m, uint32_t j, float t) {
    constexpr int H = kLearnH;
    const __nv_bfloat16* w = m.w;
    float in[kLearnIn];
    in[0] = t;
#pragma unroll
    for (int q = 0; q < 4; q++) in[1 + q] = __bfloat162float(m.emb[(uint64_t)j * 4 + q]);
    float h1[H], h2[H];
    const __nv_bfloat16* W1 = w;
    const __nv_bfloat16* B1 = W1 + H * kLearnIn;
    const __nv_bfloat16* W2 = B1 + H;
    const __nv_bfloat16* B2 = W2 + H * H;
    const __nv_bfloat16* W3 = B2 + H;
    const __nv_bfloat16* B3 = W3 + H;
#pragma unroll
    for (int r = 0; r < H; r++) {
        float acc = __bfloat162float(B1[r]);
#pragma unroll
        for (int q = 0; q < kLearnIn; q++) acc = fmaf(__bfloat162float(W1[r * kLearnIn + q]), in[q], acc);
        h1[r] = fmaxf(acc, 0.f);
    }
#pragma unroll
    for (int r = 0; r < H; r++) {
        float acc = __bfloat162float(B2[r]);
#pragma unroll
        for (int q = 0; q < H; q++) acc = fmaf(__bfloat162float(W2[r * H + q]), h1[q], acc);
        h2[r] = fmaxf(acc, 0.f);
    }
    float out = __bfloat162float(B3[0]);
#pragma unroll
    for (int q = 0; q < H; q++) out = fmaf(__bfloat162float(W3[q]), h2[q], out);
    return out;
}

// Predicted offset of key k from the first position of piece j (the
// position is j * P plus this, added in integer arithmetic).
__device__ __forceinline__ float learn_predict(const LModel& m, uint32_t j, uint64_t k) {
    uint64_t kbj = __ldg(m.kb + j);
    float x = (float)(k - kbj);
    float pos = __ldg(m.pc + j) + __ldg(m.pa + j) * x;
    if (m.hidden > 0 && __ldg(m.use_mlp + j)) {
        float t = fminf(fmaxf(x * __ldg(m.pinv + j), 0.f), 1.f);
        pos += (float)m.P * learn_mlp(m, j, t);
    }
    return pos;
}

// First index p in [lo, hi) with keys[p] >= k (hi if none).
__device__ __forceinline__ uint64_t lower_bound_in(const uint64_t* keys, uint64_t lo, uint64_t hi, uint64_t k) {
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (__ldg(keys + mid) < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// lower_bound(keys, k) through the model: search the piece's error window,
// confirm keys[p-1] < k <= keys[p], else binary-search everything.
__device__ __forceinline__ uint64_t learn_lower_bound(const LModel& m, uint64_t k, bool* fell_back) {
    *fell_back = false;
    if (m.n == 0 || k <= __ldg(m.keys)) return 0;
    if (k > __ldg(m.keys + m.n - 1)) return m.n;
    uint32_t j = learn_piece(m, k);
    int64_t e = (int64_t)__ldg(m.eps + j) + 1;
    int64_t c = (int64_t)j * m.P + (int64_t)floorf(learn_predict(m, j, k));
    int64_t lo = c - e, hi = c + e + 2;
    if (lo < 1) lo = 1;
    if (hi > (int64_t)m.n) hi = (int64_t)m.n;
    if (lo < hi) {
        uint64_t p = lower_bound_in(m.keys, (uint64_t)lo, (uint64_t)hi, k);
        // keys[0] < k here, so an answer p >= 1 is confirmed by keys[p-1] < k <= keys[p]
        if (p < (uint64_t)hi && __ldg(m.keys + p - 1) < k) return p;
    }
    *fell_back = true;
    return lower_bound_in(m.keys, 0, m.n, k);
}

}  // namespace hv
