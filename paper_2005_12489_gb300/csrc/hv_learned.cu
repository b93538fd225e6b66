// Learned position index (a layer on top of HiVision's R-tree lookups,
// Sec. 3.1, with no counterpart in the paper): a piecewise-linear + MLP model
// of an object's position in the Hilbert-sorted order as a function of its
// key, trained on the device with the kernels below, with a per-piece error
// bound measured over every key.  Objects with extent are found through their
// centre key within a halo; the few whose half-extent exceeds the halo go to
// a small side R-tree.
#include <math.h>

#include "hv_device.cuh"
#include "hv_internal.h"
#include "hv_learned.cuh"

namespace hv {

int build_side_tree(Ctx* c, int4* objs, uint32_t* ids, uint64_t n, Tree* t, int4** sorted_objs,
                    uint32_t** sorted_ids);

namespace {

constexpr int kDefaultHidden = kLearnH;
constexpr int kDefaultSteps = 300;
constexpr int kBatch = 1 << 16;

uint32_t blocks_for(uint64_t n, int t) { return (uint32_t)((n + t - 1) / t); }

struct Alloc {
    Learned* l;
    Ctx* c;
    int get(void** p, uint64_t bytes) {
        int rc = dev_alloc(c, p, bytes ? bytes : 16);
        if (rc == HV_OK) l->allocs.push_back({*p, bytes ? bytes : 16});
        return rc;
    }
};

__global__ void k_piece_first(const uint64_t* keys, uint64_t n, uint32_t P, uint32_t n_seg, uint64_t* kb) {
    uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (j < n_seg) kb[j] = keys[j * P];
}

// Radix table: rt[t] = number of pieces whose first key is < t << 46.
__global__ void k_radix(const uint64_t* kb, uint32_t n_seg, uint32_t* rt) {
    uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t > (1u << kRadixBits) + 1) return;
    uint64_t bound = t << (62 - kRadixBits);
    uint32_t lo = 0, hi = n_seg;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (kb[mid] < bound) lo = mid + 1; else hi = mid;
    }
    rt[t] = lo;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Least-squares line per piece in the normalised coordinate t in [0, 1]:
// one warp per piece, positions relative to the piece start.
__global__ void k_fit(const uint64_t* keys, uint64_t n, const uint64_t* kb, uint32_t n_seg, uint32_t P,
                      float* pa, float* pc, float* pinv) {
    uint64_t j = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (j >= n_seg) return;
    uint64_t i0 = j * P, i1 = i0 + P < n ? i0 + P : n;
    uint64_t k0 = kb[j];
    uint64_t k1 = j + 1 < n_seg ? kb[j + 1] : keys[n - 1] + 1;
    double span = (double)(k1 - k0);
    double inv = span > 0 ? 1.0 / span : 0.0;
    double st = 0, sy = 0, stt = 0, sty = 0;
    for (uint64_t i = i0 + lane; i < i1; i += 32) {
        double t = (double)(keys[i] - k0) * inv;
        double y = (double)(i - i0);
        st += t; sy += y; stt += t * t; sty += t * y;
    }
    st = warp_sum_d(st); sy = warp_sum_d(sy); stt = warp_sum_d(stt); sty = warp_sum_d(sty);
    if (lane == 0) {
        double N = (double)(i1 - i0);
        double var = stt - st * st / N;
        double a = var > 1e-30 ? (sty - st * sy / N) / var : 0.0;
        double c = (sy - a * st) / N;
        pa[j] = (float)(a * inv);
        pc[j] = (float)c;
        pinv[j] = (float)inv;
    }
}

// Deterministic small initial weights.
__device__ __forceinline__ float hash_uniform(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
    return (float)(x >> 40) * (1.0f / 16777216.0f) - 0.5f;
}

__global__ void k_init(float* w, int nw, int H, uint32_t seed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    // W1 and W2 random (fan-in scaled), biases and the output layer zero:
    // the model starts as the piecewise-linear fit alone.
    int w1 = H * kLearnIn, w2s = w1 + H, w2e = w2s + H * H;
    float v = 0.f;
    if (i < w1) v = hash_uniform(seed * 7919ull + i) * 2.0f / sqrtf((float)kLearnIn);
    else if (i >= w2s && i < w2e) v = hash_uniform(seed * 7919ull + i) * 2.0f / sqrtf((float)H);
    w[i] = v;
}

__global__ void k_to_bf16(const float* src, __nv_bfloat16* dst, uint64_t n) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16(src[i]);
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// One training step on kBatch sampled keys: forward with the fp32 master
// weights, squared error against the residual of the linear piece, backward;
// gradients warp-reduced, then accumulated in shared and global memory.
__global__ void k_train(LModel m, const float* w, const float* emb, float* gw, float* gemb, int step, uint32_t seed) {
    __shared__ float sg[kLearnNW];
    constexpr int H = kLearnH;
    constexpr int nw = kLearnNW;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) sg[i] = 0.f;
    __syncthreads();
    uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t h = ((uint64_t)seed << 32) ^ ((uint64_t)step * 0x9E3779B97F4A7C15ull) ^ (gid * 0xD1B54A32D192ED03ull);
    h ^= h >> 31; h *= 0x94D049BB133111EBull; h ^= h >> 29;
    uint64_t i = h % m.n;
    uint64_t k = m.keys[i];
    uint32_t j = learn_piece(m, k);
    uint64_t kbj = m.kb[j];
    float x = (float)(k - kbj);
    float lin = m.pc[j] + m.pa[j] * x;
    float target = ((float)((double)i - (double)j * m.P) - lin) / (float)m.P;
    float in[kLearnIn];
    in[0] = fminf(fmaxf(x * m.pinv[j], 0.f), 1.f);
    for (int q = 0; q < 4; q++) in[1 + q] = emb[(uint64_t)j * 4 + q];
    const float* W1 = w;
    const float* B1 = W1 + H * kLearnIn;
    const float* W2 = B1 + H;
    const float* B2 = W2 + H * H;
    const float* W3 = B2 + H;
    const float* B3 = W3 + H;
    float h1[H], h2[H], d2[H], d1[H];
    for (int r = 0; r < H; r++) {
        float acc = B1[r];
        for (int q = 0; q < kLearnIn; q++) acc = fmaf(W1[r * kLearnIn + q], in[q], acc);
        h1[r] = fmaxf(acc, 0.f);
    }
    for (int r = 0; r < H; r++) {
        float acc = B2[r];
        for (int q = 0; q < H; q++) acc = fmaf(W2[r * H + q], h1[q], acc);
        h2[r] = fmaxf(acc, 0.f);
    }
    float out = B3[0];
    for (int q = 0; q < H; q++) out = fmaf(W3[q], h2[q], out);
    float dout = 2.f * (out - target) / (float)kBatch;
    for (int r = 0; r < H; r++) d2[r] = h2[r] > 0.f ? dout * W3[r] : 0.f;
    for (int q = 0; q < H; q++) {
        float acc = 0.f;
        for (int r = 0; r < H; r++) acc = fmaf(d2[r], W2[r * H + q], acc);
        d1[q] = h1[q] > 0.f ? acc : 0.f;
    }
    // embedding gradient (input features 1..4): a piece's embedding sees about
    // one sample per step, so it takes the per-sample gradient, not the batch
    // mean the shared weights take
    for (int q = 1; q < kLearnIn; q++) {
        float acc = 0.f;
        for (int r = 0; r < H; r++) acc = fmaf(d1[r], W1[r * kLearnIn + q], acc);
        atomicAdd(gemb + (uint64_t)j * 4 + (q - 1), acc * (float)kBatch);
    }
    int lane = threadIdx.x & 31;
    int idx = 0;
#define HV_ACC(val)                                  \
    {                                                \
        float v_ = warp_sum_f(val);                  \
        if (lane == 0) atomicAdd(sg + idx, v_);      \
        idx++;                                       \
    }
#pragma unroll 1
    for (int r = 0; r < H; r++)
        for (int q = 0; q < kLearnIn; q++) HV_ACC(d1[r] * in[q]);
#pragma unroll 1
    for (int r = 0; r < H; r++) HV_ACC(d1[r]);
#pragma unroll 1
    for (int r = 0; r < H; r++)
        for (int q = 0; q < H; q++) HV_ACC(d2[r] * h1[q]);
    for (int r = 0; r < H; r++) HV_ACC(d2[r]);
    for (int q = 0; q < H; q++) HV_ACC(dout * h2[q]);
    HV_ACC(dout);
#undef HV_ACC
    __syncthreads();
    for (int t = threadIdx.x; t < nw; t += blockDim.x) atomicAdd(gw + t, sg[t]);
}

__global__ void k_adam(float* w, float* g, float* mo, float* ve, int nw, int step, float lr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    const float b1 = 0.9f, b2 = 0.999f;
    float gi = g[i];
    mo[i] = b1 * mo[i] + (1 - b1) * gi;
    ve[i] = b2 * ve[i] + (1 - b2) * gi * gi;
    float mh = mo[i] / (1 - powf(b1, (float)(step + 1)));
    float vh = ve[i] / (1 - powf(b2, (float)(step + 1)));
    w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
    g[i] = 0.f;
}

__global__ void k_sgd(float* w, float* g, uint64_t n, float lr) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    w[i] -= lr * g[i];
    g[i] = 0.f;
}

// Per-piece error bound over every stored key, measured with the inference
// code the lookups use.
__global__ void k_eps(LModel m, uint32_t* eps, unsigned long long* sum_err) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    float e = 0.f;
    if (i < m.n) {
        uint64_t k = m.keys[i];
        uint32_t j = learn_piece(m, k);
        float within = learn_predict(m, j, k);
        int64_t c = (int64_t)j * m.P + (int64_t)floorf(within);
        int64_t d = (int64_t)i - c;
        if (d < 0) d = -d;
        atomicMax(eps + j, (uint32_t)(d > 0xfffffff0ll ? 0xfffffff0ll : d));
        e = fabsf(within - (float)((int64_t)i - (int64_t)j * m.P));
    }
    // mean absolute error, for reporting
    unsigned long long s = (unsigned long long)e;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum_err, s);
}

// max and sum of the per-piece bounds (out[0] = max, out[1] = sum)
// Keep the MLP term for a piece only where it narrows the piece's bound.
__global__ void k_choose(const uint32_t* eps_lin, uint32_t* eps, uint8_t* use, uint32_t n_seg) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_seg) return;
    bool u = eps[j] < eps_lin[j];
    use[j] = u ? 1 : 0;
    if (!u) eps[j] = eps_lin[j];
}

__global__ void k_count_u8(const uint8_t* a, uint32_t n, unsigned long long* out) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v = (j < n && a[j]) ? 1u : 0u;
    v = __reduce_add_sync(kFull, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

__global__ void k_fill_u8(uint8_t* a, uint32_t n, uint8_t v) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) a[j] = v;
}

__global__ void k_max_u32(const uint32_t* a, uint32_t n, unsigned long long* out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t v = i < n ? a[i] : 0u;
    uint32_t mx = __reduce_max_sync(kFull, v);
    unsigned long long sm = v;
    for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(kFull, sm, o);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)mx);
        atomicAdd(out + 1, sm);
    }
}

// Half-extent of each record's box (half the larger side, plus one) and a
// histogram of its bit length; boxes are read at boxes[i * stride].
__global__ void k_extent_hist(const int4* boxes, uint32_t stride, uint64_t n, unsigned long long* hist) {
    // per-block counts in shared memory, one global add per bin and block
    __shared__ unsigned int hs[65];
    for (int k = threadIdx.x; k < 65; k += blockDim.x) hs[k] = 0u;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        int4 b = boxes[i * stride];
        if (b.x > b.z) continue;  // empty box
        int64_t w = (int64_t)b.z - b.x, h = (int64_t)b.w - b.y;
        int64_t e = (w > h ? w : h) / 2 + 1;
        atomicAdd(&hs[64 - __clzll((unsigned long long)e)], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 65; k += blockDim.x)
        if (hs[k]) atomicAdd(hist + k, (unsigned long long)hs[k]);
}

__global__ void k_mark_outliers(const int4* boxes, uint32_t stride, uint64_t n, int64_t halo, uint32_t* flag,
                                unsigned long long* count) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 b = boxes[i * stride];
    bool out = false;
    if (b.x <= b.z) {
        int64_t w = (int64_t)b.z - b.x, h = (int64_t)b.w - b.y;
        out = (w > h ? w : h) / 2 + 1 > halo;
    }
    flag[i] = out ? 1u : 0u;
    if (out) atomicAdd(count, 1ull);
}

__global__ void k_collect(const int4* boxes, const uint32_t* ids, uint64_t n, const uint32_t* flag, int4* out,
                          uint32_t* out_ids, unsigned long long* pos) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    unsigned long long p = atomicAdd(pos, 1ull);
    out[p] = boxes[i];
    out_ids[p] = ids ? ids[i] : (uint32_t)i;
}

}  // namespace

// Build the model over sorted keys `keys[0..n)` (objects `obj` of `kind`).
// boxes: the records' boxes at boxes[i * stride] (NULL for points: no
// extent).  With allow_outliers the halo covers 99.5% of the records and the
// rest go to a side tree (only for plain box records, stride 1); otherwise the
// halo covers every record.
static int build_one(Ctx* c, Learned* L, const uint64_t* keys, uint64_t n, const int4* boxes, uint32_t stride,
                     bool allow_outliers, const uint32_t* ids, const hv_build_opts* opts, int64_t* err_out) {
    Alloc A{L, c};
    LearnedView& v = L->view;
    v = LearnedView();
    v.n_obj = n;
    v.keys = keys;
    if (n == 0) { v.ready = true; return HV_OK; }
    uint32_t P = 512;
    if (opts && opts->learned_segments) {
        uint64_t p = (n + opts->learned_segments - 1) / opts->learned_segments;
        P = (uint32_t)(p < 1 ? 1 : (p > (1u << 20) ? (1u << 20) : p));
    }
    uint32_t n_seg = (uint32_t)((n + P - 1) / P);
    // the MLP has a fixed width (kLearnH); learned_hidden = 0 keeps the default,
    // any other value enables it as well
    const int H = kDefaultHidden;
    int steps = opts && opts->learned_steps ? (int)opts->learned_steps : kDefaultSteps;
    if (opts && opts->learned_hidden == HV_LEARNED_NO_MLP) steps = 0;   // linear pieces only
    uint32_t seed = opts ? opts->learned_seed : 0;
    uint64_t *kb;
    float *pa, *pc, *pinv;
    uint32_t *eps, *rt;
    HV_TRY(A.get((void**)&kb, (uint64_t)n_seg * 8));
    HV_TRY(A.get((void**)&pa, (uint64_t)n_seg * 4));
    HV_TRY(A.get((void**)&pc, (uint64_t)n_seg * 4));
    HV_TRY(A.get((void**)&pinv, (uint64_t)n_seg * 4));
    HV_TRY(A.get((void**)&eps, (uint64_t)n_seg * 4));
    HV_TRY(A.get((void**)&rt, ((1u << kRadixBits) + 2) * 4));
    k_piece_first<<<blocks_for(n_seg, 256), 256>>>(keys, n, P, n_seg, kb);
    k_radix<<<blocks_for((1u << kRadixBits) + 2, 256), 256>>>(kb, n_seg, rt);
    k_fit<<<blocks_for((uint64_t)n_seg * 32, 256), 256>>>(keys, n, kb, n_seg, P, pa, pc, pinv);
    HV_CUDA(cudaGetLastError());
    LModel m;
    m.keys = keys; m.n = n; m.kb = kb; m.pa = pa; m.pc = pc; m.pinv = pinv; m.eps = eps; m.rt = rt;
    m.emb = nullptr; m.w = nullptr; m.use_mlp = nullptr; m.n_seg = n_seg; m.P = P; m.hidden = 0;
    // error of the linear pieces alone
    unsigned long long* scratch;
    HV_TRY(dev_alloc(c, (void**)&scratch, 64));
    // max bound, mean |error|, and the sum of per-piece bounds (the average
    // search window, what a lookup pays)
    auto measure = [&](const LModel& mm, uint32_t* max_eps, double* mean, double* sum_eps) -> int {
        cudaMemset(eps, 0, (uint64_t)n_seg * 4);
        cudaMemset(scratch, 0, 64);
        k_eps<<<blocks_for(n, 256), 256>>>(mm, eps, scratch);
        k_max_u32<<<blocks_for(n_seg, 256), 256>>>(eps, n_seg, scratch + 1);
        unsigned long long h[3];
        cudaError_t e = cudaMemcpy(h, scratch, 24, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { set_error("learned error pass: %s", cudaGetErrorString(e)); return HV_ECUDA; }
        *mean = (double)h[0] / (double)n;
        *max_eps = (uint32_t)h[1];
        *sum_eps = (double)h[2];
        return HV_OK;
    };
    uint32_t eps_lin = 0, eps_mlp = 0, eps_fin = 0;
    double mean_lin = 0, mean_mlp = 0, sum_lin = 0, sum_mlp = 0, mean_fin = 0, sum_fin = 0;
    uint8_t* use;
    uint32_t* eps_l;
    HV_TRY(A.get((void**)&use, n_seg));
    HV_TRY(A.get((void**)&eps_l, (uint64_t)n_seg * 4));
    k_fill_u8<<<blocks_for(n_seg, 256), 256>>>(use, n_seg, 0);
    m.use_mlp = use;
    int rc = measure(m, &eps_lin, &mean_lin, &sum_lin);
    if (rc != HV_OK) { dev_free(c, scratch, 64); return rc; }
    HV_CUDA(cudaMemcpy(eps_l, eps, (uint64_t)n_seg * 4, cudaMemcpyDeviceToDevice));
    eps_fin = eps_lin; mean_fin = mean_lin; sum_fin = sum_lin;
    // MLP residual, trained on the device
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0);
    int nw = H * kLearnIn + H + H * H + H + H + 1;
    float *w, *gw, *mo, *ve, *emb, *gemb;
    __nv_bfloat16 *wb, *embb;
    bool ok = A.get((void**)&w, nw * 4) == HV_OK && A.get((void**)&gw, nw * 4) == HV_OK &&
              A.get((void**)&mo, nw * 4) == HV_OK && A.get((void**)&ve, nw * 4) == HV_OK &&
              A.get((void**)&emb, (uint64_t)n_seg * 16) == HV_OK && A.get((void**)&gemb, (uint64_t)n_seg * 16) == HV_OK &&
              A.get((void**)&wb, nw * 2) == HV_OK && A.get((void**)&embb, (uint64_t)n_seg * 8) == HV_OK;
    uint32_t pieces_mlp = 0;
    if (ok && steps > 0 && H > 0) {
        cudaMemset(gw, 0, nw * 4);
        cudaMemset(mo, 0, nw * 4);
        cudaMemset(ve, 0, nw * 4);
        cudaMemset(emb, 0, (uint64_t)n_seg * 16);
        cudaMemset(gemb, 0, (uint64_t)n_seg * 16);
        k_init<<<blocks_for(nw, 256), 256>>>(w, nw, H, seed + 1);
        LModel tm = m;
        tm.hidden = H;
        for (int s = 0; s < steps; s++) {
            k_train<<<kBatch / 256, 256>>>(tm, w, emb, gw, gemb, s, seed);
            k_adam<<<blocks_for(nw, 256), 256>>>(w, gw, mo, ve, nw, s, 2e-3f);
            k_sgd<<<blocks_for((uint64_t)n_seg * 4, 256), 256>>>(emb, gemb, (uint64_t)n_seg * 4, 0.02f);
        }
        k_to_bf16<<<blocks_for(nw, 256), 256>>>(w, wb, nw);
        k_to_bf16<<<blocks_for((uint64_t)n_seg * 4, 256), 256>>>(emb, embb, (uint64_t)n_seg * 4);
        HV_CUDA(cudaGetLastError());
        // every piece with the MLP term ...
        LModel mm = m;
        mm.hidden = H;
        mm.w = wb;
        mm.emb = embb;
        k_fill_u8<<<blocks_for(n_seg, 256), 256>>>(use, n_seg, 1);
        rc = measure(mm, &eps_mlp, &mean_mlp, &sum_mlp);
        if (rc != HV_OK) { dev_free(c, scratch, 64); return rc; }
        // ... then each piece keeps the model with the narrower bound, and the
        // bounds are measured again with the combined model
        k_choose<<<blocks_for(n_seg, 256), 256>>>(eps_l, eps, use, n_seg);
        rc = measure(mm, &eps_fin, &mean_fin, &sum_fin);
        if (rc != HV_OK) { dev_free(c, scratch, 64); return rc; }
        unsigned long long* cntd = scratch + 4;
        HV_CUDA(cudaMemset(cntd, 0, 8));
        k_count_u8<<<blocks_for(n_seg, 256), 256>>>(use, n_seg, cntd);
        unsigned long long hc = 0;
        HV_CUDA(cudaMemcpy(&hc, cntd, 8, cudaMemcpyDeviceToHost));
        pieces_mlp = (uint32_t)hc;
        if (pieces_mlp) m = mm;
    }
    cudaEventRecord(t1);
    cudaEventSynchronize(t1);
    float ms = 0;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    L->train_ms += ms;
    if (!pieces_mlp) {
        k_fill_u8<<<blocks_for(n_seg, 256), 256>>>(use, n_seg, 0);
        rc = measure(m, &eps_fin, &mean_fin, &sum_fin);  // the linear bounds alone
        if (rc != HV_OK) { dev_free(c, scratch, 64); return rc; }
    }
    dev_free(c, scratch, 64);
    v.seg_a = pa;
    v.seg_b = pc;
    v.seg_k0 = kb;
    v.radix = rt;
    v.mlp = (const uint16_t*)m.w;
    v.emb = (const uint16_t*)m.emb;
    v.use_mlp = use;
    v.pinv = pinv;
    v.eps_piece = eps;
    v.n_seg = n_seg;
    v.P = P;
    v.hidden = m.hidden;
    v.eps = eps_fin;
    v.eps_linear = eps_lin;
    v.eps_mlp = eps_mlp;
    v.mean_err = mean_fin;
    v.mean_err_linear = mean_lin;
    v.mean_window = sum_fin / (double)n_seg;
    v.mean_window_linear = sum_lin / (double)n_seg;
    v.pieces_mlp = pieces_mlp;
    *err_out = v.eps;
    // halo and side tree for objects with extent
    if (boxes) {
        unsigned long long* hist;
        HV_TRY(dev_alloc(c, (void**)&hist, 65 * 8));
        cudaMemset(hist, 0, 65 * 8);
        k_extent_hist<<<(unsigned)(blocks_for(n, 256) < 4096 ? blocks_for(n, 256) : 4096), 256>>>(boxes, stride, n,
                                                                                                hist);
        unsigned long long hh[65];
        cudaError_t e = cudaMemcpy(hh, hist, 65 * 8, cudaMemcpyDeviceToHost);
        dev_free(c, hist, 65 * 8);
        if (e != cudaSuccess) { set_error("extent histogram: %s", cudaGetErrorString(e)); return HV_ECUDA; }
        uint64_t total = 0, acc = 0;
        for (int b = 0; b < 65; b++) total += hh[b];
        int bits = 0;
        for (int b = 0; b < 65; b++) {
            acc += hh[b];
            if (allow_outliers ? acc * 1000 >= total * 995 : acc == total) { bits = b; break; }
        }
        int64_t halo = bits >= 31 ? ((int64_t)1 << 31) : ((int64_t)1 << bits);
        v.halo = (int32_t)(halo > 0x7fffffff ? 0x7fffffff : halo);
        uint32_t* flag;
        unsigned long long* cnt;
        HV_TRY(dev_alloc(c, (void**)&flag, n * 4));
        HV_TRY(dev_alloc(c, (void**)&cnt, 16));
        cudaMemset(cnt, 0, 16);
        k_mark_outliers<<<blocks_for(n, 256), 256>>>(boxes, stride, n, v.halo, flag, cnt);
        unsigned long long n_out = 0;
        HV_CUDA(cudaMemcpy(&n_out, cnt, 8, cudaMemcpyDeviceToHost));
        L->n_outliers = n_out;
        if (n_out) {
            int4* oo;
            uint32_t* oid;
            rc = dev_alloc(c, (void**)&oo, n_out * 16);
            if (rc == HV_OK) rc = dev_alloc(c, (void**)&oid, n_out * 4);
            if (rc != HV_OK) { dev_free(c, flag, n * 4); dev_free(c, cnt, 16); return rc; }
            cudaMemset(cnt + 1, 0, 8);
            k_collect<<<blocks_for(n, 256), 256>>>(boxes, ids, n, flag, oo, oid, cnt + 1);
            HV_CUDA(cudaGetLastError());
            int4* so;
            uint32_t* sid;
            rc = build_side_tree(c, oo, oid, n_out, &L->outlier_tree, &so, &sid);
            if (rc != HV_OK) { dev_free(c, flag, n * 4); dev_free(c, cnt, 16); return rc; }
            L->allocs.push_back({so, n_out * 16});
            L->allocs.push_back({sid, n_out * 4});
            v.outliers = L->outlier_tree.view;
            v.outlier_obj = so;
            v.outlier_ids = sid;
        }
        dev_free(c, flag, n * 4);
        dev_free(c, cnt, 16);
    }
    HV_CUDA(cudaDeviceSynchronize());
    v.ready = true;
    return HV_OK;
}

int build_learned(Layer* L, const hv_build_opts* opts) {
    Ctx* c = L->ctx;
    uint32_t max_err = opts && opts->max_error ? opts->max_error : 4096;
    int64_t e1 = 0, e2 = 0;
    // segment pieces: their boxes follow each segment in the record, and the
    // bounded piece extent makes every record fit the halo (no side tree)
    const int4* piece_boxes = L->kind == HV_LAYER_POINTS ? nullptr : (const int4*)L->obj + 1;
    HV_TRY(build_one(c, &L->learned, L->keys, L->n_obj, piece_boxes, 2, false, nullptr, opts, &e1));
    if (L->kind == HV_LAYER_POLYGONS)
        HV_TRY(build_one(c, &L->mbr_learned, L->mbr_keys, L->n_poly, L->mbr_obj, 1, true, L->mbr_ids, opts, &e2));
    if ((uint64_t)e1 > max_err || (uint64_t)e2 > max_err) {
        set_error("learned index rejected: position error bound %lld exceeds %u",
                  (long long)(e1 > e2 ? e1 : e2), max_err);
        free_learned(c, &L->learned);
        free_learned(c, &L->mbr_learned);
        return HV_ESTATE;
    }
    return HV_OK;
}

void free_learned(Ctx* c, Learned* l) {
    for (auto& a : l->allocs) dev_free(c, a.first, a.second);
    l->allocs.clear();
    free_tree(c, &l->outlier_tree);
    l->view = LearnedView();
    l->n_outliers = 0;
}

// ---- lookups for the C ABI (tests, diagnostics) -----------------------------

namespace {
__global__ void k_lookup(LModel m, const uint64_t* q, uint32_t n, uint64_t* out, unsigned long long* fallbacks) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool fb;
    out[i] = learn_lower_bound(m, q[i], &fb);
    if (fb) atomicAdd(fallbacks, 1ull);
}
}  // namespace

LModel learned_model(const LearnedView& v) {
    LModel m;
    m.keys = v.keys;
    m.n = v.n_obj;
    m.kb = v.seg_k0;
    m.pa = v.seg_a;
    m.pc = v.seg_b;
    m.pinv = v.pinv;
    m.eps = v.eps_piece;
    m.rt = v.radix;
    m.emb = (const __nv_bfloat16*)v.emb;
    m.w = (const __nv_bfloat16*)v.mlp;
    m.use_mlp = v.use_mlp;
    m.n_seg = v.n_seg;
    m.P = v.P;
    m.hidden = v.hidden;
    return m;
}

int learned_lookup(Layer* L, int which, const uint64_t* q, uint32_t n, uint64_t* out, uint64_t* fallbacks,
                   cudaStream_t st) {
    const Learned& l = which == 0 ? L->learned : L->mbr_learned;
    if (!l.view.ready) { set_error("learned index not built"); return HV_ESTATE; }
    unsigned long long* fb;
    HV_TRY(dev_alloc(L->ctx, (void**)&fb, 8));
    cudaMemsetAsync(fb, 0, 8, st);
    if (n) k_lookup<<<blocks_for(n, 256), 256, 0, st>>>(learned_model(l.view), q, n, out, fb);
    cudaError_t e = cudaMemcpyAsync(fallbacks, fb, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(L->ctx, fb, 8);
    if (e != cudaSuccess) { set_error("learned lookup: %s", cudaGetErrorString(e)); return HV_ECUDA; }
    return HV_OK;
}

}  // namespace hv
