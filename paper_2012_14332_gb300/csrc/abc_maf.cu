// abc_maf.cu -- masked autoregressive flow proposal for sequential ABC:
// density, sampling (sequential inverse), weighted maximum-likelihood
// gradient and Adam, with BF16 tensor-core products (mma.sync m16n8k8 and
// m16n8k16 per warp tile; tcgen05.mma with TMEM accumulators for the weight
// gradients; FP32 accumulation).
//
// A warp owns 16 rows (samples). A row's eight coordinates sit in the
// accumulator layout of an m16n8 tile: lane (g = lane / 4, t = lane % 4) holds
// columns 2t, 2t+1 of rows g and g+8. That is also the A-operand layout of an
// m16n8k8 product, so a MADE block runs entirely in registers:
//   layer 1  a1 = x W1^T + b1  : per 16 hidden units two m16n8k8 products;
//   layer 2  out = relu(a1) W2^T + b2 : the two layer-1 accumulator tiles are
//            exactly the A fragment of one m16n8k16 step, so the hidden layer
//            never leaves registers (16 units at a time).
// The order reversal between blocks (column j <-> 7 - j) is a shuffle with
// lane ^ 3; row sums are shuffles over the 4 lanes of a row.
// Weight gradients reduce over rows: their products take the warps' operands
// from shared memory on tcgen05 and accumulate in tensor memory per CTA.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <random>
#include <utility>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/abc_gb300.h"
#include "abc_kernels.h"
#include "abc_model.cuh"

namespace abcgb {
abc_status plan_fail(abc_status st, const char* msg);
abc_status plan_cuda_fail(cudaError_t e, const char* what);
abc_status plan_ok();
bool plan_check_prior(const abc_prior_box* prior, abc_status* st);
ModelParams plan_make_params(const abc_prior_box* prior, int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream,
                             const int32_t* ard0);

namespace maf {

constexpr int kHMax = 256;
constexpr int kKMax = 4;
constexpr float kAlphaMax = 6.0f;
constexpr uint32_t kFull = 0xFFFFFFFFu;

// Master (FP32) parameters of one block: W1 [H][8], b1 [H], W2 [16][H], b2 [16].
__host__ __device__ inline int master_block(int H) { return 25 * H + 16; }

// Published BF16 layout of one block, in 32-bit words (two bf16 per word).
// The forward operands come first, so density and sampling kernels stage only
// fwd_words per block; the gradient kernel stages all words. The forward
// operands are grouped by 16-unit hidden chunk s and lane (g = lane / 4,
// t = lane % 4) so that one chunk's fragments are one vector load per lane:
//   w1  [H/16][8][4][2]  B operands of x W1^T (k = input j = 2t, 2t+1) for
//                        hidden units 16s + g and 16s + 8 + g
//   w2  [H/16][8][4][4]  B operands of h W2^T (k = hidden 16s + 2t, +1 and
//                        16s + 8 + 2t, +1) for outputs g and 8 + g
//   b1  [H/16][4][4]     FP32: b1 of hidden 16s + 2t, +1, 16s + 8 + 2t, +1
//   b2  [16]             FP32
//   w1t [8][H/2+4]       B operand of g_a1 W1     (n = j, k = l)
//   w2t [H][8]           B operand of g_out W2    (n = l, k = o); rows l with
//                        l & 4 hold their two 4-word halves swapped, so the
//                        warp's fragment loads meet 32 distinct banks
// then the sampler's copy of the forward operands (sw1, sw2, sb1 in the w1,
// w2, b1 layouts, and sb2 = b2), whose 16-unit chunks hold the hidden units
// grouped by degree: every degree d = 1..7 has the same number of chunks,
// sampler_cpd(H) (the chunks degree 1, which has the most units, needs),
// holding units d - 1, d + 6, d + 13, ... in order, padded with zero units.
struct Layout {
    int w1, w2, b1, b2, w1t, w2t, fwd_words, grad_words;
    int sw1, sw2, sb1, sb2, samp_words, words;
};

// MADE masks (Germain et al.): hidden degree (l mod 7) + 1; input j and output
// j (mu_j and alpha_j, o = j and o = 8 + j) have degree j + 1.
__host__ __device__ inline bool mask1(int l, int j) { return (l % 7) + 1 >= j + 1; }
__host__ __device__ inline bool mask2(int o, int l) { return (o % 8) + 1 > (l % 7) + 1; }

// hidden units of degree d (1..7) among H, and the 16-unit chunks they fill
__host__ __device__ inline int degree_units(int H, int d) { return (H - d) / 7 + 1; }
__host__ __device__ inline int degree_chunks(int H, int d) { return (degree_units(H, d) + 15) / 16; }
// chunks per degree in the sampler's copy (1 up to H = 112, 2 up to 224, 3 up to 256)
__host__ __device__ inline int sampler_cpd(int H) { return degree_chunks(H, 1); }
__host__ __device__ inline int sampler_chunks(int H) { return 7 * sampler_cpd(H); }
// hidden unit at position u (0..15) of sampler chunk s, or -1 for padding
__host__ __device__ inline int sampler_unit(int H, int s, int u)
{
    const int cpd = sampler_cpd(H), d = s / cpd + 1, i = 16 * (s % cpd) + u;
    return i < degree_units(H, d) ? d - 1 + 7 * i : -1;
}

__host__ __device__ inline Layout layout(int H)
{
    Layout L;
    int o = 0;
    L.w1 = o; o += H * 4;
    L.w2 = o; o += H * 8;
    L.b1 = o; o += H;
    L.b2 = o; o += 16;
    L.fwd_words = o;
    L.w1t = o; o += 8 * (H / 2 + 4);
    L.w2t = o; o += H * 8;
    L.grad_words = o;
    const int C = sampler_chunks(H);
    L.sw1 = o; o += C * 64;
    L.sw2 = o; o += C * 128;
    L.sb1 = o; o += C * 16;
    L.sb2 = o; o += 16;
    L.samp_words = o - L.sw1;
    L.words = o;
    return L;
}

struct Box {
    float lo[8], w[8], logw[8];
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// bf16x2 of (max(lo, 0), max(hi, 0)), round to nearest: the ReLU folded into
// the conversion (for a negative input the rounded value is <= 0 and clamps
// to 0, as clamping first would give)
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_k16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                        uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// The same products as plain asm (no side effects): the compiler may
// interleave independent chains, which the gradient kernel's backward pass
// uses to overlap neighbouring chunks.
__device__ __forceinline__ void mma_k8_p(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0)
{
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_k16_p(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                          uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct BlockView {
    const uint32_t* w1;
    const uint32_t* w2;
    const uint32_t* w1t;
    const uint32_t* w2t;
    const float* b1;
    const float* b2;
};

__device__ __forceinline__ BlockView view(const uint32_t* base, const Layout& L)
{
    BlockView v;
    v.w1 = base + L.w1;
    v.w2 = base + L.w2;
    v.w1t = base + L.w1t;
    v.w2t = base + L.w2t;
    v.b1 = reinterpret_cast<const float*>(base + L.b1);
    v.b2 = reinterpret_cast<const float*>(base + L.b2);
    return v;
}

__device__ __forceinline__ float quad_sum(float v)
{
    v += __shfl_xor_sync(kFull, v, 1);
    v += __shfl_xor_sync(kFull, v, 2);
    return v;
}

// column j <-> 7 - j within each row (accumulator layout)
__device__ __forceinline__ void reverse_cols(float (&v)[4])
{
    const float n0 = __shfl_xor_sync(kFull, v[1], 3), n1 = __shfl_xor_sync(kFull, v[0], 3);
    const float n2 = __shfl_xor_sync(kFull, v[3], 3), n3 = __shfl_xor_sync(kFull, v[2], 3);
    v[0] = n0; v[1] = n1; v[2] = n2; v[3] = n3;
}

// alpha = A tanh(ar / A) from one exponential: tanh|y| = (1 - e) / (1 + e) with
// e = exp(-2 |y|) in (0, 1], so nothing overflows; the fast exponential and
// division leave an absolute error of a few 1e-7 in alpha
__device__ __forceinline__ float soft_alpha(float ar)
{
    const float e = __expf((-2.f / kAlphaMax) * fabsf(ar));
    return copysignf(kAlphaMax * __fdividef(1.f - e, 1.f + e), ar);
}

// Density and sampling CTAs: 8 warps share one staged copy of the forward
// operands (about 41 KB at 3 x 256), at most 64 registers so that 4 CTAs
// (32 warps) fit on an SM to hide the tensor-core chains' latency.
constexpr int kFwdThreads = 256;
constexpr int kFwdMinBlocks = 4;
// The sampler's longer passes run better at 3 CTAs per SM (80 registers,
// 16 bytes spilled, against 64 and 32): 1.182 -> 1.157 ms per 0.9 x 2^22
// proposals at 3 x 256.
constexpr int kSampMinBlocks = 3;

// The base density: independent standard logistic coordinates,
// log p(z) = -|z| - 2 log(1 + exp(-|z|)); d(-log p)/dz = tanh(z / 2). The logit
// of a uniform variable is standard logistic, so the flow with zero
// parameters is the uniform prior on the box.
// The flow's transcendentals outside the products use the SFU forms
// (__expf, __logf, __fdividef): their absolute errors of about 1e-7 are far
// inside the flow's BF16 accuracy, and the density is always evaluated at
// the point actually produced, so the proposal stays self-consistent.
__device__ __forceinline__ float log_base(float z)
{
    const float a = fabsf(z);
    return -a - 2.f * __logf(1.f + __expf(-a));
}

// a standard logistic draw from one random word: logit of its uniform u in
// (0, 1); u = (2m + 1) 2^-24, so 1 - u is exact
__device__ __forceinline__ float logistic_draw(uint32_t w)
{
    const float u = uniform01(w);
    return __logf(u) - __logf(1.f - u);
}

// One 16-unit hidden chunk of a MADE on the warp's 16 rows: layer 1 (two
// m16n8k8, accumulators starting at b1), ReLU and bf16 in one conversion,
// then the chunk's layer-2 contribution (two m16n8k16) into o0 (mu) and o1
// (alpha_raw).
__device__ __forceinline__ void made_chunk(const BlockView& v, int s, int g, int t, uint32_t a0, uint32_t a1,
                                           float (&o0)[4], float (&o1)[4])
{
    const uint2 wa = reinterpret_cast<const uint2*>(v.w1)[(s * 8 + g) * 4 + t];
    const uint4 wb = reinterpret_cast<const uint4*>(v.w2)[(s * 8 + g) * 4 + t];
    const float4 bb = reinterpret_cast<const float4*>(v.b1)[s * 4 + t];
    float c0[4] = {bb.x, bb.y, bb.x, bb.y}, c1[4] = {bb.z, bb.w, bb.z, bb.w};
    mma_k8(c0, a0, a1, wa.x);
    mma_k8(c1, a0, a1, wa.y);
    const uint32_t A0 = pack2_relu(c0[0], c0[1]), A1 = pack2_relu(c0[2], c0[3]);
    const uint32_t A2 = pack2_relu(c1[0], c1[1]), A3 = pack2_relu(c1[2], c1[3]);
    mma_k16(o0, A0, A1, A2, A3, wb.x, wb.y);
    mma_k16(o1, A0, A1, A2, A3, wb.z, wb.w);
}

// One MADE on the warp's 16 rows: mu and alpha_raw in the accumulator layout.
// Even and odd chunks accumulate separately (two independent tensor-core
// chains), summed at the end.
__device__ __forceinline__ void made_fwd(const BlockView& v, int H, const float (&x)[4], float (&mu)[4],
                                         float (&ar)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t a0 = pack2(x[0], x[1]), a1 = pack2(x[2], x[3]);
    float o0[4] = {0.f, 0.f, 0.f, 0.f}, o1[4] = {0.f, 0.f, 0.f, 0.f};
    float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
    const int chunks = H / 16;
    int s = 0;
    for (; s + 1 < chunks; s += 2) {
        made_chunk(v, s, g, t, a0, a1, o0, o1);
        made_chunk(v, s + 1, g, t, a0, a1, p0, p1);
    }
    if (s < chunks) made_chunk(v, s, g, t, a0, a1, o0, o1);
    const float2 bm = *reinterpret_cast<const float2*>(v.b2 + 2 * t);
    const float2 bs = *reinterpret_cast<const float2*>(v.b2 + 8 + 2 * t);
    mu[0] = (o0[0] + p0[0]) + bm.x; mu[1] = (o0[1] + p0[1]) + bm.y;
    mu[2] = (o0[2] + p0[2]) + bm.x; mu[3] = (o0[3] + p0[3]) + bm.y;
    ar[0] = (o1[0] + p1[0]) + bs.x; ar[1] = (o1[1] + p1[1]) + bs.y;
    ar[2] = (o1[2] + p1[2]) + bs.x; ar[3] = (o1[3] + p1[3]) + bs.y;
}

// The partial MADE outputs (without b2) of hidden chunks [s0, s1) on the
// warp's 16 rows: the contributions to mu and alpha_raw, even and odd chunks in
// separate chains added at the end.
__device__ __forceinline__ void made_part(const BlockView& v, int s0, int s1, const float (&x)[4], float (&pm)[4],
                                          float (&pa)[4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint32_t a0 = pack2(x[0], x[1]), a1 = pack2(x[2], x[3]);
    float o0[4] = {0.f, 0.f, 0.f, 0.f}, o1[4] = {0.f, 0.f, 0.f, 0.f};
    float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
    int s = s0;
    for (; s + 1 < s1; s += 2) {
        made_chunk(v, s, g, t, a0, a1, o0, o1);
        made_chunk(v, s + 1, g, t, a0, a1, p0, p1);
    }
    if (s < s1) made_chunk(v, s, g, t, a0, a1, o0, o1);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        pm[e] = o0[e] + p0[e];
        pa[e] = o1[e] + p1[e];
    }
}

// theta -> y = logit((theta - lo) / w) and the log-Jacobian term log(w u (1 - u)).
// u is held in [2^-24, 1 - 2^-24]: a point on the box's edge (a flow draw whose
// sigmoid rounded to 0 or 1) is read as lying 2^-24 of the width inside.
__device__ __forceinline__ void to_y(const Box& b, int j, float th, float& y, float& jac)
{
    const float u = fminf(fmaxf((th - b.lo[j]) / b.w[j], 0x1p-24f), 0x1.fffffep-1f);
    const float lu = __logf(u), l1u = __logf(1.f - u);
    y = lu - l1u;
    jac = b.logw[j] + lu + l1u;
}

// y -> theta = lo + w sigmoid(y) and log(w s (1 - s)).
__device__ __forceinline__ void to_theta(const Box& b, int j, float y, float& th, float& jac)
{
    const float e = __expf(-fabsf(y));
    const float l = __logf(1.f + e);
    const float ls = fminf(y, 0.f) - l, l1s = fminf(-y, 0.f) - l;
    const float s = __fdividef(y >= 0.f ? 1.f : e, 1.f + e);
    th = b.lo[j] + b.w[j] * s;
    jac = b.logw[j] + ls + l1s;
}

// words [off, off + n) of each of K published blocks, packed block after
// block in shared memory (stride n). Every offset and length is a multiple of
// 4 words (H is a multiple of 16), so the copy moves 16-byte vectors.
__device__ __forceinline__ void stage_blocks(uint32_t* sm, const uint32_t* pub, int K, int off, int n,
                                             const Layout& L)
{
    const int n4 = n / 4;
    for (int i = threadIdx.x; i < K * n4; i += blockDim.x) {
        const int b = i / n4, r = i - b * n4;
        reinterpret_cast<uint4*>(sm)[i] = reinterpret_cast<const uint4*>(pub + (size_t)b * L.words + off)[r];
    }
}

// ---------------------------------------------------------------------------
// publish: masked BF16 copies (and biases) from the FP32 master parameters
// ---------------------------------------------------------------------------
// Every word of each block's published operands, padding included (a
// training step's Adam launch republishes the parameters it updates, one
// parameter per thread, and never writes the padding).
__global__ void publish_kernel(const float* __restrict__ master, uint32_t* __restrict__ pub, int K, int H)
{
    const Layout L = layout(H);
    const int per = L.words, limit = L.words, mb = master_block(H), hw = H / 2 + 4;
    master += (size_t)blockIdx.y * K * mb;   // flow blockIdx.y
    pub += (size_t)blockIdx.y * K * per;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * limit; i += gridDim.x * blockDim.x) {
        const int b = i / limit, w = i % limit, idx = b * per + w;
        const float* M = master + (size_t)b * mb;
        const float* W1 = M;
        const float* b1 = M + 8 * H;
        const float* W2 = M + 9 * H;
        const float* b2 = M + 25 * H;
        uint32_t out = 0;
        if (w < L.w2) {
            // r = ((s 8 + g) 4 + t) 2 + h: hidden l = 16 s + g + 8 h, inputs 2t, 2t+1
            const int r = w - L.w1, h = r & 1, t = (r >> 1) & 3, g = (r >> 3) & 7, sc = r >> 6;
            const int l = 16 * sc + g + 8 * h, j0 = 2 * t;
            __nv_bfloat162 v = __floats2bfloat162_rn(mask1(l, j0) ? W1[l * 8 + j0] : 0.f,
                                                     mask1(l, j0 + 1) ? W1[l * 8 + j0 + 1] : 0.f);
            out = *reinterpret_cast<uint32_t*>(&v);
        } else if (w < L.b1) {
            // r = ((s 8 + g) 4 + t) 4 + q: output g + 8 (q / 2), hidden 16 s + 8 (q % 2) + 2t, +1
            const int r = w - L.w2, q = r & 3, t = (r >> 2) & 3, g = (r >> 4) & 7, sc = r >> 7;
            const int o = g + 8 * (q >> 1), l0 = 16 * sc + 8 * (q & 1) + 2 * t;
            __nv_bfloat162 v = __floats2bfloat162_rn(mask2(o, l0) ? W2[o * H + l0] : 0.f,
                                                     mask2(o, l0 + 1) ? W2[o * H + l0 + 1] : 0.f);
            out = *reinterpret_cast<uint32_t*>(&v);
        } else if (w < L.b2) {
            // r = (s 4 + t) 4 + q: b1 of hidden 16 s + 8 (q / 2) + 2t + q % 2
            const int r = w - L.b1, q = r & 3, t = (r >> 2) & 3, sc = r >> 4;
            out = __float_as_uint(b1[16 * sc + 8 * (q >> 1) + 2 * t + (q & 1)]);
        } else if (w < L.w1t) {
            out = __float_as_uint(b2[w - L.b2]);
        } else if (w < L.w2t) {
            const int r = w - L.w1t, j = r / hw, c = r % hw;
            if (c < H / 2) {
                const int l0 = 2 * c;
                __nv_bfloat162 v = __floats2bfloat162_rn(mask1(l0, j) ? W1[l0 * 8 + j] : 0.f,
                                                         mask1(l0 + 1, j) ? W1[(l0 + 1) * 8 + j] : 0.f);
                out = *reinterpret_cast<uint32_t*>(&v);
            }
        } else if (w < L.grad_words) {
            const int r = w - L.w2t, l = r / 8, o0 = 2 * ((r % 8) ^ (l & 4));
            __nv_bfloat162 v = __floats2bfloat162_rn(mask2(o0, l) ? W2[o0 * H + l] : 0.f,
                                                     mask2(o0 + 1, l) ? W2[(o0 + 1) * H + l] : 0.f);
            out = *reinterpret_cast<uint32_t*>(&v);
        } else if (w < L.sw2) {
            // as w1, over the degree-grouped chunks: unit at position g + 8 h of chunk s
            const int r = w - L.sw1, h = r & 1, t = (r >> 1) & 3, g = (r >> 3) & 7, sc = r >> 6;
            const int l = sampler_unit(H, sc, g + 8 * h), j0 = 2 * t;
            __nv_bfloat162 v = __floats2bfloat162_rn(l >= 0 && mask1(l, j0) ? W1[l * 8 + j0] : 0.f,
                                                     l >= 0 && mask1(l, j0 + 1) ? W1[l * 8 + j0 + 1] : 0.f);
            out = *reinterpret_cast<uint32_t*>(&v);
        } else if (w < L.sb1) {
            const int r = w - L.sw2, q = r & 3, t = (r >> 2) & 3, g = (r >> 4) & 7, sc = r >> 7;
            const int o = g + 8 * (q >> 1), u0 = 8 * (q & 1) + 2 * t;
            const int l0 = sampler_unit(H, sc, u0), l1 = sampler_unit(H, sc, u0 + 1);
            __nv_bfloat162 v = __floats2bfloat162_rn(l0 >= 0 && mask2(o, l0) ? W2[o * H + l0] : 0.f,
                                                     l1 >= 0 && mask2(o, l1) ? W2[o * H + l1] : 0.f);
            out = *reinterpret_cast<uint32_t*>(&v);
        } else if (w < L.sb2) {
            const int r = w - L.sb1, q = r & 3, t = (r >> 2) & 3, sc = r >> 4;
            const int l = sampler_unit(H, sc, 8 * (q >> 1) + 2 * t + (q & 1));
            out = __float_as_uint(l >= 0 ? b1[l] : 0.f);
        } else {
            out = __float_as_uint(b2[w - L.sb2]);
        }
        pub[idx] = out;
    }
}

// ---------------------------------------------------------------------------
// density: log q(theta)
// ---------------------------------------------------------------------------
// The proposal may use a broadened base, z = tau * (standard logistic), with
// density log p(z / tau) - log tau per coordinate (tau = 1: the trained flow).
template <int K>
__global__ void __launch_bounds__(kFwdThreads, kFwdMinBlocks) logq_kernel(const uint32_t* __restrict__ pub, int H, Box box,
                                                   const float* __restrict__ theta, uint64_t n, float inv_tau,
                                                   float log_tau, float* __restrict__ logq)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const Layout L = layout(H);
    stage_blocks(sm, pub, K, 0, L.fwd_words, L);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint64_t tiles = (n + 15) / 16;
    const int warps = blockDim.x / 32;
    for (uint64_t tile = (uint64_t)blockIdx.x * warps + (threadIdx.x >> 5); tile < tiles;
         tile += (uint64_t)gridDim.x * warps) {
        const uint64_t r0 = tile * 16 + g, r1 = r0 + 8;
        float x[4], jac[4];
        const float mid[2] = {box.lo[2 * t] + 0.5f * box.w[2 * t], box.lo[2 * t + 1] + 0.5f * box.w[2 * t + 1]};
        const float2 ta = r0 < n ? *reinterpret_cast<const float2*>(theta + 8 * r0 + 2 * t) : make_float2(mid[0], mid[1]);
        const float2 tb = r1 < n ? *reinterpret_cast<const float2*>(theta + 8 * r1 + 2 * t) : make_float2(mid[0], mid[1]);
        to_y(box, 2 * t, ta.x, x[0], jac[0]);
        to_y(box, 2 * t + 1, ta.y, x[1], jac[1]);
        to_y(box, 2 * t, tb.x, x[2], jac[2]);
        to_y(box, 2 * t + 1, tb.y, x[3], jac[3]);
        float ld[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b < K; ++b) {
            float mu[4], ar[4];
            made_fwd(view(sm + b * L.fwd_words, L), H, x, mu, ar);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float al = soft_alpha(ar[e]);
                x[e] = (x[e] - mu[e]) * __expf(-al);
                ld[e] -= al;
            }
            reverse_cols(x);
        }
        const float q0 = quad_sum(log_base(x[0] * inv_tau) + log_base(x[1] * inv_tau) + ld[0] + ld[1] - jac[0] -
                                  jac[1] - 2.f * log_tau);
        const float q1 = quad_sum(log_base(x[2] * inv_tau) + log_base(x[3] * inv_tau) + ld[2] + ld[3] - jac[2] -
                                  jac[3] - 2.f * log_tau);
        if (t == 0) {
            if (r0 < n) logq[r0] = q0;
            if (r1 < n) logq[r1] = q1;
        }
    }
}

// One pass of the sequential inverse: the CPD chunks of degree-D hidden units
// (chunks (D-1) CPD .. D CPD - 1 of the sampler's copy). Their inputs (columns
// below D) are all final, so each unit's activation is computed once, and its
// layer-2 contribution to every output is added to the running accumulators
// (even chunks into o, odd into p). D and CPD are compile-time, so every
// operand load is a fixed offset from the lane's base in the block's copy.
template <int D, int CPD>
__device__ __forceinline__ void inverse_pass(const BlockView& v, int g, int t, const float (&xin)[4], float (&o0)[4],
                                             float (&o1)[4], float (&p0)[4], float (&p1)[4])
{
    const uint32_t a0 = pack2(xin[0], xin[1]), a1 = pack2(xin[2], xin[3]);
#pragma unroll
    for (int c = 0; c < CPD; ++c) {
        const int s = (D - 1) * CPD + c;
        if (s & 1)
            made_chunk(v, s, g, t, a0, a1, p0, p1);
        else
            made_chunk(v, s, g, t, a0, a1, o0, o1);
    }
}

// Column D of the block's inverse, once pass D has added every unit of degree
// <= D: lane t = D / 2 holds it, element D % 2 for row g and 2 + D % 2 for row g + 8.
template <int D>
__device__ __forceinline__ void inverse_column(int t, const float (&z)[4], float (&xin)[4], float (&lq)[4],
                                               const float (&o0)[4], const float (&o1)[4], const float (&p0)[4],
                                               const float (&p1)[4])
{
    constexpr int e = D & 1;
    if (t == D / 2) {
        const float al0 = soft_alpha(o1[e] + p1[e]), al1 = soft_alpha(o1[2 + e] + p1[2 + e]);
        xin[e] = z[e] * __expf(al0) + (o0[e] + p0[e]);
        xin[2 + e] = z[2 + e] * __expf(al1) + (o0[2 + e] + p0[2 + e]);
        lq[e] -= al0;
        lq[2 + e] -= al1;
    }
}

template <int D, int CPD>
__device__ __forceinline__ void inverse_passes(const BlockView& v, int g, int t, const float (&z)[4], float (&xin)[4],
                                               float (&lq)[4], float (&o0)[4], float (&o1)[4], float (&p0)[4],
                                               float (&p1)[4])
{
    if constexpr (D <= 7) {
        inverse_pass<D, CPD>(v, g, t, xin, o0, o1, p0, p1);
        inverse_column<D>(t, z, xin, lq, o0, o1, p0, p1);
        inverse_passes<D + 1, CPD>(v, g, t, z, xin, lq, o0, o1, p0, p1);
    }
}

template <int K, int CPD>
// box: read in place from the parameter space (indexing a by-value copy by
// the lane's column put it in local memory)
__global__ void __launch_bounds__(kFwdThreads, kSampMinBlocks) sample_kernel(const uint32_t* __restrict__ pub, int H,
                                                     const __grid_constant__ Box box,
                                                     const float* __restrict__ u_in, const __grid_constant__ ModelParams p,
                                                     uint32_t ctr3, uint64_t first, uint64_t n, float tau,
                                                     float log_tau, float* __restrict__ theta_out,
                                                     float* __restrict__ logq_out)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const Layout L = layout(H);
    stage_blocks(sm, pub, K, L.sw1, L.samp_words, L);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint64_t tiles = (n + 15) / 16;
    const int warps = blockDim.x / 32;
    for (uint64_t tile = (uint64_t)blockIdx.x * warps + (threadIdx.x >> 5); tile < tiles;
         tile += (uint64_t)gridDim.x * warps) {
        const uint64_t r0 = tile * 16 + g, r1 = r0 + 8;
        float x[4];
        if (u_in) {
            const float2 ua = r0 < n ? *reinterpret_cast<const float2*>(u_in + 8 * r0 + 2 * t) : make_float2(0.f, 0.f);
            const float2 ub = r1 < n ? *reinterpret_cast<const float2*>(u_in + 8 * r1 + 2 * t) : make_float2(0.f, 0.f);
            x[0] = ua.x; x[1] = ua.y; x[2] = ub.x; x[3] = ub.y;
        } else {
            // row r: Philox block (t / 2) of sample first + r; lane t takes words
            // (x, y) for even t and (z, w) for odd t, one word per column
            const uint4 wa = rng_block_s(p, first + r0, 0, ctr3, (uint32_t)(t >> 1));
            const uint4 wb = rng_block_s(p, first + r1, 0, ctr3, (uint32_t)(t >> 1));
            x[0] = logistic_draw((t & 1) ? wa.z : wa.x);
            x[1] = logistic_draw((t & 1) ? wa.w : wa.y);
            x[2] = logistic_draw((t & 1) ? wb.z : wb.x);
            x[3] = logistic_draw((t & 1) ? wb.w : wb.y);
        }
        float lq[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            lq[e] = log_base(x[e]) - log_tau;
            x[e] *= tau;
        }
        // blocks are a runtime loop (a fully unrolled 3 x 7 inverse overflows
        // the instruction cache); a block's seven passes are unrolled, so
        // every operand offset and register index is static. Column j
        // depends on the hidden units of degree <= j alone, which passes
        // 1..j have added to the accumulators by then.
#pragma unroll 1
        for (int bb = K - 1; bb >= 0; --bb) {
            const uint32_t* base = sm + bb * L.samp_words;
            BlockView v;
            v.w1 = base;
            v.w2 = base + (L.sw2 - L.sw1);
            v.b1 = reinterpret_cast<const float*>(base + (L.sb1 - L.sw1));
            v.b2 = reinterpret_cast<const float*>(base + (L.sb2 - L.sw1));
            v.w1t = v.w2t = nullptr;
            float z[4] = {x[0], x[1], x[2], x[3]};
            reverse_cols(z);
            float xin[4] = {0.f, 0.f, 0.f, 0.f};
            const float2 bm = *reinterpret_cast<const float2*>(v.b2 + 2 * t);
            const float2 bs = *reinterpret_cast<const float2*>(v.b2 + 8 + 2 * t);
            float o0[4] = {bm.x, bm.y, bm.x, bm.y}, o1[4] = {bs.x, bs.y, bs.x, bs.y};
            float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
            if (t == 0) {
                // column 0 has degree 1: every weight into mu_0, alpha_0 is masked
                const float al0 = soft_alpha(bs.x);
                xin[0] = z[0] * __expf(al0) + bm.x;
                xin[2] = z[2] * __expf(al0) + bm.x;
                lq[0] -= al0;
                lq[2] -= al0;
            }
            inverse_passes<1, CPD>(v, g, t, z, xin, lq, o0, o1, p0, p1);
            x[0] = xin[0]; x[1] = xin[1]; x[2] = xin[2]; x[3] = xin[3];
        }
        float th[4], jac[4];
        to_theta(box, 2 * t, x[0], th[0], jac[0]);
        to_theta(box, 2 * t + 1, x[1], th[1], jac[1]);
        to_theta(box, 2 * t, x[2], th[2], jac[2]);
        to_theta(box, 2 * t + 1, x[3], th[3], jac[3]);
        const float q0 = quad_sum(lq[0] + lq[1] - jac[0] - jac[1]);
        const float q1 = quad_sum(lq[2] + lq[3] - jac[2] - jac[3]);
        if (r0 < n) *reinterpret_cast<float2*>(theta_out + 8 * r0 + 2 * t) = make_float2(th[0], th[1]);
        if (r1 < n) *reinterpret_cast<float2*>(theta_out + 8 * r1 + 2 * t) = make_float2(th[2], th[3]);
        if (t == 0 && logq_out) {
            if (r0 < n) logq_out[r0] = q0;
            if (r1 < n) logq_out[r1] = q1;
        }
    }
}

// ---------------------------------------------------------------------------
// gradient of sum_r w_r (-log q_y(y_r)) (unnormalised; Adam divides by sum w)
// ---------------------------------------------------------------------------
// The forward pass and the backward products of each row (g_h = g_out W2,
// g_x = g_a1 W1) run in the warp's registers on mma.sync, as in the density
// kernel. The weight gradients reduce over rows:
//   dW2^T [l][o]       = sum over rows of h[row][l] g_out[row][o]
//   [dW1 | db1] [l][j] = sum over rows of g_a1[row][l] [x | 1][row][j]
// (j < 8: dW1, j = 8: db1). Per warp tile both are products of M = 128 hidden
// units x N = 16 x K = 16 rows. They run on the tensor cores (tcgen05.mma,
// BF16 operands from shared memory, FP32 accumulators in tensor memory) and
// accumulate over every tile the CTA processes: TMEM lane = hidden unit within
// a 128-unit half, 16 columns per product and (block, half). The CTA adds its
// sums to the flow's gradient once, at the end.
//
// Warps 0..W-1 compute; one lane of warp W issues the products. A compute
// warp's job is one (block, half) of one tile: it stores h and g_a1 of 128
// hidden units (eight 16-unit chunks) into its A slot (and, in a block's
// first job, g_out and x into its B slot), then arrives on full[w]. The
// issuing thread takes round n (job n of every warp) in warp order, issues
// each job's two products and commits the round to one round barrier. A
// warp waits for its previous round's phase of that barrier before the first
// store of its next job; a commit tracks every product the thread issued
// before it, so the previous block's products are done when the B slot is
// rewritten. All products come from one thread in issue order, so
// accumulations into the same TMEM columns never race.
//
// Operands in shared memory are MN-major (hidden unit, output or input
// contiguous), without swizzle: a core matrix is 8 rows of k (tile rows) x 16
// bytes (8 bf16 along m or n); core matrices 128 bytes apart along K (the
// descriptor's leading byte offset) and 256 bytes apart along M or N (stride
// byte offset). Lane (g, t) of the accumulator layout holds columns 2t, 2t+1
// of rows g and g + 8: one 32-bit word at byte 16 g + 4 t of a core matrix,
// so a warp's 32 stores meet 32 distinct banks.
//
// In the paired form (PAIR, two 128-unit halves) warps 2p and 2p + 1 share a
// tile: member m recomputes and differentiates only the hidden units of half
// m, so its job per block is the (block, m) pair, and the two add their
// partial layer-2 outputs (forward) and partial g_x (backward) through shared
// memory once per block. A tile's dependent chain is then half as long, and a
// CTA holds two tiles instead of four, so a small batch spreads over twice
// as many SMs.
//
// Every wait is bounded in time (kTcWaitNs). A wait that runs out sets the
// flow's error word; the kernel still runs to its end and frees its TMEM.
//
// The gradient is reproducible bit for bit: the issuing thread takes the
// compute warps' jobs in a fixed order (job n of warp 0, 1, ..., W-1, then job
// n + 1), so the tensor-memory accumulations into each column group happen in
// the same order in every run; db2 and the loss sums collect per warp and add
// up in warp order; in the paired form the two members add their partial
// sums commutatively, so both hold the same values; and each CTA writes its
// whole partial gradient to its own slot of a buffer whose slots are added in
// a fixed tree (grad_reduce_kernel, adam_publish_kernel; no float atomics
// anywhere).

// compute warps per CTA: 4, or 15 when a step has enough tiles for more than
// two waves of 4-warp CTAs (one CTA fits per SM; 16 warps in all keep 128
// registers per thread)
constexpr int kGradWarpsNarrow = 4;
constexpr int kGradWarpsWide = 15;
constexpr int kTcM = 128;                          // hidden units per product
constexpr int kTcHalf = 4096;                      // one A operand: 128 units x 16 rows, bf16
constexpr int kTcB = 1024;                         // the B slot: g_out (512 B), [x | 1] (512 B)
constexpr int kTcSlot = 2 * kTcHalf + kTcB;        // shared memory per compute warp
constexpr uint32_t kTcLBO = 128, kTcSBO = 256;
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5), BF16 A
// and B (bits 7-9, 10-12), both MN-major (bits 15, 16), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28)
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((16u >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);
constexpr unsigned long long kTcWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void st_u32(unsigned char* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

// has the phase of this parity completed (no waiting)
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// waits for the phase of this parity to complete, for at most kTcWaitNs. The
// clock (a long-latency read of the global timer) starts only once a first
// try has failed, and is read every 8th try after that: the issuing thread
// meets mostly completed phases, and a timer read per wait had cost it
// hundreds of cycles per job.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 7u) == 0 && global_ns() - t0 > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// this thread's shared-memory stores become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(kTcLBO >> 4) << 16) | ((uint64_t)(kTcSBO >> 4) << 32) |
           (1ull << 46);
}

// D (TMEM) = A B + (accumulate ? D : 0)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d), "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
                 : "memory");
}

// arrives on the barrier once every product this thread issued has completed
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (lane i: thread i)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr)
                 : "memory");
}

// 32 consecutive 32-bit columns of this warp's 32 TMEM lanes (lane i: thread i)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr)
                 : "memory");
}

// one hidden unit's dW1 row (eight inputs, masked) as two 16-byte stores
__device__ __forceinline__ void store_dw1(float* __restrict__ row, int l, const uint32_t* v)
{
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = mask1(l, j) ? __uint_as_float(v[j]) : 0.f;
    float4* r4 = reinterpret_cast<float4*>(row);
    r4[0] = make_float4(w[0], w[1], w[2], w[3]);
    r4[1] = make_float4(w[4], w[5], w[6], w[7]);
}

// mbarrier arrival that also adds `bytes` to the transaction count of the
// current phase (the bytes bulk copies will complete on it)
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// bulk copy (no tensor map) of `bytes` from global to this CTA's shared
// memory, completing on the mbarrier; both addresses and the size are
// multiples of 16 bytes
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// The K blocks' words [off, off + n) of the published operands, copied into
// sm (K x n words, packed) by the bulk-copy engine: thread 0 sets the
// barrier's transaction count and issues one copy per block. The barrier was
// initialised (count 1) and that made visible to the CTA before the call.
// Offsets and sizes are multiples of 4 words (16 bytes), as the bulk copy
// requires: every section of the layout is, since H is a multiple of 16.
__device__ __forceinline__ void stage_blocks_bulk(uint32_t* sm, const uint32_t* pub, int K, int off, int n,
                                                  const Layout& L, uint32_t bar)
{
    if (threadIdx.x != 0) return;
    mbar_arrive_expect_tx(bar, (uint32_t)(K * n) * 4u);
    for (int b = 0; b < K; ++b) bulk_g2s(smem_addr(sm + b * n), pub + (size_t)b * L.words + off, (uint32_t)n * 4u, bar);
}

// The two warps of a pair add their partial sums: each stores its N values per
// lane in its half of the exchange buffer for this parity, waits on the pair's
// named barrier (64 threads), and adds the other warp's values. Float addition
// is commutative, so both warps end with the same sums bit for bit. Two
// parities: a warp rewrites a buffer only after the next exchange's barrier,
// which the other warp reaches after it read the buffer.
template <int N>
__device__ __forceinline__ void pair_add(float* __restrict__ buf, uint32_t& xc, int member, int bar_id, int lane,
                                         float (&v)[N])
{
    float* mine = buf + ((xc & 1u) * 2 + member) * (8 * 32);
    const float* other = buf + ((xc & 1u) * 2 + (member ^ 1)) * (8 * 32);
#pragma unroll
    for (int e = 0; e < N; ++e) mine[32 * e + lane] = v[e];
    asm volatile("bar.sync %0, 64;" ::"r"(bar_id) : "memory");
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] += other[32 * e + lane];
    ++xc;
}

// Row b of flow f's training batch at step `step`: a uniform draw, with
// replacement, from the flow's n points (one Philox block per row).
__device__ __forceinline__ uint32_t batch_row(const ModelParams& p, uint32_t b, uint32_t step, int f, uint64_t n)
{
    const uint4 w = philox10(make_uint4(b, step, 0xB47C4u, 0x5EEDu + ((uint32_t)f << 16)), p);
    return (uint32_t)((((uint64_t)w.y << 32) | w.x) % n);
}

// Training data of one flow: points theta [n][8], weights [n] (NULL = 1).
struct TrainSlot {
    const float* theta;
    const float* w;
    uint64_t n;
};

// The rows of one tile for lane (g, t): sample indices, weights and the
// lane's two coordinates of rows q0 = 16 tile + g and q1 = q0 + 8 (rows past
// n_rows: weight 0, row 0's data). With a ticket (a training step) the rows
// are batch_row draws, lanes t = 0 and 1 of the row group drawing q0 and q1.
// Called by the whole warp.
struct TileRows {
    float w0, w1;
    float2 ta, tb;
};

__device__ __forceinline__ TileRows tile_rows(uint64_t tile, int g, int t, int lane, uint64_t n_rows, bool drawn,
                                              const ModelParams& rp, uint32_t step, int f, const TrainSlot& slot)
{
    const uint64_t q0 = tile * 16 + g, q1 = q0 + 8;
    uint64_t i0 = q0 < n_rows ? q0 : 0, i1 = q1 < n_rows ? q1 : 0;
    if (drawn) {
        const uint64_t qm = t ? q1 : q0;
        const uint32_t mine = t < 2 && qm < n_rows ? batch_row(rp, (uint32_t)qm, step, f, slot.n) : 0u;
        i0 = __shfl_sync(kFull, mine, lane & ~3);
        i1 = __shfl_sync(kFull, mine, (lane & ~3) | 1);
    }
    TileRows r;
    r.w0 = q0 < n_rows ? (slot.w ? slot.w[i0] : 1.f) : 0.f;
    r.w1 = q1 < n_rows ? (slot.w ? slot.w[i1] : 1.f) : 0.f;
    r.ta = *reinterpret_cast<const float2*>(slot.theta + 8 * i0 + 2 * t);
    r.tb = *reinterpret_cast<const float2*>(slot.theta + 8 * i1 + 2 * t);
    return r;
}

// Flow f = blockIdx.y reads slots[f]: with a ticket counter (a training step),
// `batch` rows drawn for the step (batch_row; none if the flow has no points),
// else all its n points. Each CTA of a training launch takes a ticket; the
// step is the ticket over `ctas`, the launch's CTA count, whatever order the
// CTAs start in, and after the launch the counter stands at (step + 1) ctas.
// Dynamic shared memory: W slots of kTcSlot bytes, then the K blocks' published
// operands.
template <int K, int W, bool PAIR>
__global__ void __launch_bounds__((W + 1) * 32, 1) grad_kernel(const uint32_t* __restrict__ pub, int H,
                                                               const __grid_constant__ Box box,
                                                               const TrainSlot* __restrict__ slots,
                                                               unsigned* __restrict__ ticket, uint32_t ctas,
                                                               const __grid_constant__ ModelParams rp, uint32_t batch,
                                                               float* __restrict__ part, uint32_t part_stride,
                                                               int* __restrict__ err, int hold)
{
    static_assert(W >= 4 && W <= 15, "at least one compute warp per TMEM lane quarter; 16 warps in all at most");
    static_assert(!PAIR || W % 2 == 0, "whole pairs");
    constexpr int TPC = PAIR ? W / 2 : W;   // tiles a CTA works on at once
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[W], bar_round, bar_done, bar_stage;
    __shared__ uint32_t tmem_s, init_s;
    __shared__ float ssum_w[W][2];       // per compute warp: weighted loss sum, weight sum
    __shared__ float gb2_w[W][K * 16];   // per compute warp: db2 sums
    __shared__ float xch[PAIR ? W / 2 : 1][2 * 2 * 8 * 32];   // per pair: parity, member, value, lane
    const Layout L = layout(H);
    const int mb = master_block(H);
    const int f = blockIdx.y;
    const TrainSlot slot = slots[f];
    __shared__ uint32_t step_s;
    if (ticket && threadIdx.x == 0) step_s = atomicAdd(ticket, 1u) / ctas;   // before any CTA returns
    const uint64_t n_rows = ticket ? (slot.n ? batch : 0) : slot.n;
    if (n_rows == 0) {   // uniform over the block
        // even a CTA with no rows completes only after the previous kernel of
        // the stream, so this launch's completion implies that kernel's
        griddep_wait();
        return;
    }
    pub += (size_t)f * K * L.words;
    // this CTA's partial: K blocks of mb parameters, then the two loss sums
    float* __restrict__ out_part = part + ((size_t)f * gridDim.x + blockIdx.x) * part_stride;
    uint32_t* wsm = reinterpret_cast<uint32_t*>(smem + W * kTcSlot);
    // the published operands arrive by bulk copy while the CTA sets up
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar_stage), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t step_now = ticket ? step_s : 0u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = (H + kTcM - 1) / kTcM;   // jobs (128-unit halves) per block
    const int D = K * C;                   // (block, half) accumulator pairs, 32 columns each
    const uint32_t ncols = D <= 1 ? 32u : D <= 2 ? 64u : D <= 4 ? 128u : 256u;
    if (warp < W) {
        // columns 8..15 of [x | 1] in the B slot: 1 in column 8, 0 after it
        unsigned char* sb = smem + warp * kTcSlot + 2 * kTcHalf + 512 + 256;
        for (int i = lane; i < 64; i += 32) st_u32(sb + 4 * i, (i & 3) == 0 ? 0x3F80u : 0u);
        fence_async_smem();
    } else {
        if (lane == 0) {
            for (int i = 0; i < W; ++i) {
                mbar_init(smem_addr(&bar_full[i]), 1);
            }
            mbar_init(smem_addr(&bar_round), 1);
            mbar_init(smem_addr(&bar_done), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_s)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = threadIdx.x; i < W * K * 16; i += blockDim.x) (&gb2_w[0][0])[i] = 0.f;
    for (int i = threadIdx.x; i < W * 2; i += blockDim.x) (&ssum_w[0][0])[i] = 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint64_t tiles = (n_rows + 15) / 16;
    const uint64_t tstride = (uint64_t)gridDim.x * TPC;
    // Up to here nothing depends on the previous kernel of the stream (in a
    // training step, the previous step's Adam, which reads the ticket before
    // it releases this launch): the set-up and the first tile's rows overlap
    // it. The published operands and the partials wait for its completion.
    const uint64_t tile0 = (uint64_t)blockIdx.x * TPC + (PAIR ? warp >> 1 : warp);
    TileRows first{};
    if (warp < W && tile0 < tiles)
        first = tile_rows(tile0, lane >> 2, lane & 3, lane, n_rows, ticket != nullptr, rp, step_now, f, slot);
    griddep_wait();
    stage_blocks_bulk(wsm, pub, K, 0, L.grad_words, L, smem_addr(&bar_stage));
    griddep_release();
    // the operands staged (a wait that runs out sets the error word; the
    // CTA's result is then not used, but it still runs to its end)
    if (!mbar_wait(smem_addr(&bar_stage), 0) && lane == 0) atomicExch(err, 1);
    const uint32_t tmem = tmem_s;
    if (warp < W) {
        const int g = lane >> 2, t = lane & 3, rg = 16 * g + 4 * t, sw = g & 4;
        unsigned char* sA = smem + warp * kTcSlot;   // h at 0, g_a1 at kTcHalf, the B slot after
        unsigned char* sB = sA + 2 * kTcHalf;
        const uint32_t full = smem_addr(&bar_full[warp]), empty = smem_addr(&bar_round);
        uint32_t job = 0;
        bool ok = true;
        const int hw = H / 2 + 4, chunks = H / 16;
        // a pair's member m takes the hidden units of half m (chunks 8m ..)
        const int pair = PAIR ? warp >> 1 : warp, member = PAIR ? warp & 1 : 0;
        const int s_lo = PAIR ? 8 * member : 0, s_hi = PAIR ? min(s_lo + 8, chunks) : chunks;
        float* xbuf = xch[PAIR ? pair : 0];
        uint32_t xc = 0;   // the pair's exchanges so far
        for (uint64_t tile = tile0; tile < tiles; tile += tstride) {
            const TileRows rows =
                tile == tile0 ? first : tile_rows(tile, g, t, lane, n_rows, ticket != nullptr, rp, step_now, f, slot);
            const float w0 = rows.w0, w1 = rows.w1;
            const float2 ta = rows.ta, tb = rows.tb;
            float x[4], jac;
            to_y(box, 2 * t, ta.x, x[0], jac);
            to_y(box, 2 * t + 1, ta.y, x[1], jac);
            to_y(box, 2 * t, tb.x, x[2], jac);
            to_y(box, 2 * t + 1, tb.y, x[3], jac);
            float xs[K][4], as[K][4], zs[K][4];
            float ld0 = 0.f, ld1 = 0.f;
#pragma unroll
            for (int b = 0; b < K; ++b) {
                float mu[4], ar[4];
                if constexpr (PAIR) {
                    const BlockView v = view(wsm + b * L.grad_words, L);
                    float pm[4], pa[4];
                    made_part(v, s_lo, s_hi, x, pm, pa);
                    float o[8] = {pm[0], pm[1], pm[2], pm[3], pa[0], pa[1], pa[2], pa[3]};
                    pair_add<8>(xbuf, xc, member, 1 + pair, lane, o);
                    const float2 bm = *reinterpret_cast<const float2*>(v.b2 + 2 * t);
                    const float2 bs = *reinterpret_cast<const float2*>(v.b2 + 8 + 2 * t);
                    mu[0] = o[0] + bm.x; mu[1] = o[1] + bm.y; mu[2] = o[2] + bm.x; mu[3] = o[3] + bm.y;
                    ar[0] = o[4] + bs.x; ar[1] = o[5] + bs.y; ar[2] = o[6] + bs.x; ar[3] = o[7] + bs.y;
                } else {
                    made_fwd(view(wsm + b * L.grad_words, L), H, x, mu, ar);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    xs[b][e] = x[e];
                    as[b][e] = soft_alpha(ar[e]);
                    zs[b][e] = (x[e] - mu[e]) * __expf(-as[b][e]);
                    x[e] = zs[b][e];
                }
                ld0 += as[b][0] + as[b][1];
                ld1 += as[b][2] + as[b][3];
                reverse_cols(x);
            }
            // nll = -log p(z) + sum alpha
            const float n0 = quad_sum(ld0 - log_base(x[0]) - log_base(x[1]));
            const float n1 = quad_sum(ld1 - log_base(x[2]) - log_base(x[3]));
            float contrib = (t == 0) ? (w0 * n0 + w1 * n1) : 0.f;
            float wsum = (t == 0) ? (w0 + w1) : 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                contrib += __shfl_xor_sync(kFull, contrib, off);
                wsum += __shfl_xor_sync(kFull, wsum, off);
            }
            if (lane == 0 && member == 0) {
                ssum_w[warp][0] += contrib;
                ssum_w[warp][1] += wsum;
            }
            // d/dz_K of sum w (-log p(z)) = w tanh(z / 2)
            float gx[4] = {w0 * tanhf(0.5f * x[0]), w0 * tanhf(0.5f * x[1]), w1 * tanhf(0.5f * x[2]),
                           w1 * tanhf(0.5f * x[3])};
            const float wr[4] = {w0, w0, w1, w1};
#pragma unroll
            for (int b = K - 1; b >= 0; --b) {
                const BlockView v = view(wsm + b * L.grad_words, L);
                reverse_cols(gx);   // gradient with respect to this block's output z
                float gmu[4], gar[4], gxd[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float ex = __expf(-as[b][e]);
                    gxd[e] = gx[e] * ex;
                    gmu[e] = -gx[e] * ex;
                    const float ga = -gx[e] * zs[b][e] + wr[e];
                    const float r = as[b][e] / kAlphaMax;
                    gar[e] = ga * (1.f - r * r);
                }
                // g_out: the A fragment of g_h = g_out W2 and, with x, this
                // block's B operands g_out [row][o] and x [row][j]
                const uint32_t A0 = pack2(gmu[0], gmu[1]), A1 = pack2(gmu[2], gmu[3]);
                const uint32_t A2 = pack2(gar[0], gar[1]), A3 = pack2(gar[2], gar[3]);
                const uint32_t xa0 = pack2(xs[b][0], xs[b][1]), xa1 = pack2(xs[b][2], xs[b][3]);
                // db2[o] = sum over rows of g_out
                {
                    float d[4] = {gmu[0] + gmu[2], gmu[1] + gmu[3], gar[0] + gar[2], gar[1] + gar[3]};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        d[e] += __shfl_xor_sync(kFull, d[e], 4);
                        d[e] += __shfl_xor_sync(kFull, d[e], 8);
                        d[e] += __shfl_xor_sync(kFull, d[e], 16);
                    }
                    if (g == 0 && member == 0) {
                        gb2_w[warp][16 * b + 2 * t] += d[0];
                        gb2_w[warp][16 * b + 2 * t + 1] += d[1];
                        gb2_w[warp][16 * b + 8 + 2 * t] += d[2];
                        gb2_w[warp][16 * b + 9 + 2 * t] += d[3];
                    }
                }
                // one 16-unit chunk; even and odd chunks keep separate g_x sums
                // (independent chains the compiler can interleave)
                auto chunk = [&](int s, float (&accx)[4]) {
                    const int q = s & 7;   // chunk within the 128-unit half
                    // recompute the pre-activations of hidden units 16s .. 16s+15
                    const uint2 wa = reinterpret_cast<const uint2*>(v.w1)[(s * 8 + g) * 4 + t];
                    const float4 bq = reinterpret_cast<const float4*>(v.b1)[s * 4 + t];
                    float c0[4] = {bq.x, bq.y, bq.x, bq.y}, c1[4] = {bq.z, bq.w, bq.z, bq.w};
                    mma_k8_p(c0, xa0, xa1, wa.x);
                    mma_k8_p(c1, xa0, xa1, wa.y);
                    // g_h = g_out W2 for these units, then through the ReLU
                    const uint32_t* w2r0 = v.w2t + (16 * s + g) * 8;
                    const uint32_t* w2r1 = w2r0 + 64;
                    float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
                    mma_k16_p(d0, A0, A1, A2, A3, w2r0[t ^ sw], w2r0[(4 ^ sw) + t]);
                    mma_k16_p(d1, A0, A1, A2, A3, w2r1[t ^ sw], w2r1[(4 ^ sw) + t]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        d0[e] = c0[e] > 0.f ? d0[e] : 0.f;
                        d1[e] = c1[e] > 0.f ? d1[e] : 0.f;
                    }
                    const uint32_t P0 = pack2(d0[0], d0[1]), P1 = pack2(d0[2], d0[3]);
                    const uint32_t P2 = pack2(d1[0], d1[1]), P3 = pack2(d1[2], d1[3]);
                    // g_x += g_a1 W1 (this chunk's 16 hidden units as k)
                    mma_k16_p(accx, P0, P1, P2, P3, v.w1t[g * hw + 8 * s + t], v.w1t[g * hw + 8 * s + 4 + t]);
                    // h and g_a1 of these units into the A slot (core matrices
                    // 2q and 2q + 1 along M); a job's first chunk waits until the
                    // products of the warp's previous job have read the slot;
                    // after one wait has run out the warp skips the rest, so a
                    // failed call returns within about one wait limit
                    if (q == 0 && job > 0 && ok) ok = mbar_wait(empty, (job - 1) & 1u);
                    if (s == s_lo) {
                        // the previous job was the previous block's last: the B slot is free
                        st_u32(sB + rg, A0);
                        st_u32(sB + 128 + rg, A1);
                        st_u32(sB + 256 + rg, A2);
                        st_u32(sB + 384 + rg, A3);
                        st_u32(sB + 512 + rg, xa0);
                        st_u32(sB + 640 + rg, xa1);
                    }
                    unsigned char* a = sA + 512 * q + rg;
                    st_u32(a, pack2_relu(c0[0], c0[1]));
                    st_u32(a + 128, pack2_relu(c0[2], c0[3]));
                    st_u32(a + 256, pack2_relu(c1[0], c1[1]));
                    st_u32(a + 384, pack2_relu(c1[2], c1[3]));
                    st_u32(a + kTcHalf, P0);
                    st_u32(a + kTcHalf + 128, P1);
                    st_u32(a + kTcHalf + 256, P2);
                    st_u32(a + kTcHalf + 384, P3);
                    if (q == 7 || s == chunks - 1) {
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(full);
                        ++job;
                    }
                };
                float ax0[4] = {0.f, 0.f, 0.f, 0.f}, ax1[4] = {0.f, 0.f, 0.f, 0.f};
                int s = s_lo;
                for (; s + 1 < s_hi; s += 2) {
                    chunk(s, ax0);
                    chunk(s + 1, ax1);
                }
                if (s < s_hi) chunk(s, ax0);
#pragma unroll
                for (int e = 0; e < 4; ++e) ax0[e] += ax1[e];
                if constexpr (PAIR) pair_add<4>(xbuf, xc, member, 1 + pair, lane, ax0);
#pragma unroll
                for (int e = 0; e < 4; ++e) gx[e] = gxd[e] + ax0[e];
            }
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    } else if (lane == 0 && hold) {
        // testing: no products, so the wait for bar_done below runs out
        init_s = 0;
    } else if (lane == 0) {
        // the issuing thread: round n is job n of every warp, issued in warp
        // order (a warp's jobs: tile, block K-1..0, half; a pair member's:
        // tile, block K-1..0, with its own half), so each column group
        // accumulates in the same order in every run. Warps whose stores are
        // already in are gathered and issued under one tensor-core fence; the
        // thread waits only on a warp that is not ready yet. One commit ends
        // the round: its products complete within about a hundred cycles,
        // and every warp waits on that round barrier before reusing its slot.
        const uint32_t per_tile = PAIR ? (uint32_t)K : (uint32_t)D;
        uint32_t total[W], most = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t t0 = (uint64_t)blockIdx.x * TPC + (PAIR ? w >> 1 : w);
            total[w] = t0 < tiles ? (uint32_t)((tiles - 1 - t0) / tstride + 1) * per_tile : 0u;
            most = total[w] > most ? total[w] : most;
        }
        uint32_t init = 0;   // accumulator pairs written at least once
        bool ok = true;
        for (uint32_t n = 0; n < most && ok; ++n) {
            const uint32_t bi = PAIR ? n : n / (uint32_t)C;   // block index in a warp's sequence
            const int b = K - 1 - (int)(bi % K), cn = PAIR ? 0 : (int)(n - bi * (uint32_t)C);
            uint32_t pending = 0;   // warps gathered, not yet issued
            auto issue = [&]() {
                tc_fence_after();
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    if (!((pending >> w) & 1u)) continue;
                    const int d = b * C + (PAIR ? (w & 1) : cn);
                    const uint32_t sa = smem_addr(smem + w * kTcSlot);
                    const uint32_t sb = sa + 2 * kTcHalf;
                    const uint32_t acc = (init >> d) & 1u;
                    init |= 1u << d;
                    tc_mma(tmem + 32 * d, tc_desc(sa), tc_desc(sb), acc);
                    tc_mma(tmem + 32 * d + 16, tc_desc(sa + kTcHalf), tc_desc(sb + 512), acc);
                }
                pending = 0;
            };
#pragma unroll
            for (int w = 0; w < W; ++w) {
                if (n >= total[w] || !ok) continue;
                const uint32_t fb = smem_addr(&bar_full[w]);
                if (!mbar_test(fb, n & 1u)) {
                    if (pending) issue();
                    if (!mbar_wait(fb, n & 1u)) {
                        atomicExch(err, 1);
                        ok = false;
                        continue;
                    }
                }
                pending |= 1u << w;
            }
            if (pending) issue();
            tc_commit(smem_addr(&bar_round));
        }
        init_s = init;
        tc_commit(smem_addr(&bar_done));
    }
    __syncthreads();
    // bar_done's first phase completes once every product of the CTA has
    const bool done = __all_sync(kFull, mbar_wait(smem_addr(&bar_done), 0));   // uniform over the warp
    if (!done && threadIdx.x == 0) atomicExch(err, 1);
    tc_fence_after();
    const uint32_t init = init_s;
    if (warp < W && done) {
        // warp w reads TMEM lanes 32 (w mod 4) .. + 31; the warps of a lane
        // quarter share its 2 D column groups. Every parameter of the CTA's
        // partial is written: masked entries and column groups this CTA never
        // accumulated (no tile) as 0.
        // A row of the partial is 16-byte aligned (its stride and the block
        // size 25 H + 16 are multiples of 4 floats, H of 16), so a unit's dW1
        // row goes out as two 16-byte stores.
        const int quarter = warp & 3, per_quarter = (W - quarter + 3) / 4;
        if (per_quarter == 1) {
            // one warp per lane quarter: both halves of a group in one load
            for (int d = 0; d < D; ++d) {
                uint32_t v[32];
                if ((init >> d) & 1u) {   // uniform over the warp
                    tc_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + 32 * d, v);
                } else {
#pragma unroll
                    for (int o = 0; o < 32; ++o) v[o] = 0u;
                }
                const int b = d / C, c = d - b * C;
                const int l = kTcM * c + 32 * quarter + lane;
                if (l >= H) continue;
                float* out = out_part + (size_t)b * mb;
#pragma unroll
                for (int o = 0; o < 16; ++o) out[9 * H + o * H + l] = mask2(o, l) ? __uint_as_float(v[o]) : 0.f;
                store_dw1(out + l * 8, l, v + 16);
                out[8 * H + l] = __uint_as_float(v[24]);
            }
        } else {
            for (int cc = warp >> 2; cc < 2 * D; cc += per_quarter) {
                const int d = cc >> 1;
                uint32_t v[16];
                if ((init >> d) & 1u) {   // uniform over the warp
                    tc_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 16 * cc, v);
                } else {
#pragma unroll
                    for (int o = 0; o < 16; ++o) v[o] = 0u;
                }
                const int b = d / C, c = d - b * C;
                const int l = kTcM * c + 32 * quarter + lane;
                if (l >= H) continue;
                float* out = out_part + (size_t)b * mb;
                if ((cc & 1) == 0) {
#pragma unroll
                    for (int o = 0; o < 16; ++o) out[9 * H + o * H + l] = mask2(o, l) ? __uint_as_float(v[o]) : 0.f;
                } else {
                    store_dw1(out + l * 8, l, v);
                    out[8 * H + l] = __uint_as_float(v[8]);
                }
            }
        }
    }
    // db2 and the loss sums: the compute warps' parts added in warp order
    for (int i = threadIdx.x; i < K * 16; i += blockDim.x) {
        float a = 0.f;
        for (int w = 0; w < W; ++w) a += gb2_w[w][i];
        out_part[(size_t)(i >> 4) * mb + 25 * H + (i & 15)] = a;
    }
    if (threadIdx.x < 2) {
        float a = 0.f;
        for (int w = 0; w < W; ++w) a += ssum_w[w][threadIdx.x];
        out_part[(size_t)K * mb + threadIdx.x] = a;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == W)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// The CTAs' partials are added in a fixed tree. A 256-thread block covers
// E = 256 / G consecutive entries in G groups: thread (q, e) adds the partials
// of CTAs q, q + G, q + 2G, ... of entry e in that order, with a chunk's loads
// all in flight at once, and the G group sums are then added in group order.
// G is the smallest of 1, 2, 4, 8 that leaves at most kRedUnroll partials per
// thread (red_groups), so a few CTAs cost one pass of loads and many CTAs
// still take about one round trip. A warp covers 32 consecutive entries: every
// load is a coalesced 128-byte row.
constexpr int kRedUnroll = 20;

template <int G>
__device__ __forceinline__ float group_sum(const float* __restrict__ q, int nblk, uint32_t stride, int grp)
{
    float a = 0.f;
    for (int c0 = grp; c0 < nblk; c0 += G * kRedUnroll) {
        float x[kRedUnroll];
#pragma unroll
        for (int k = 0; k < kRedUnroll; ++k) {
            const int c = c0 + G * k;
            x[k] = c < nblk ? q[(size_t)c * stride] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kRedUnroll; ++k) a += x[k];
    }
    return a;
}

// the same for entries e and e + off together, with both entries' loads of a
// chunk in flight at once (has0, has1: whether each entry exists)
template <int G>
__device__ __forceinline__ void group_sum2(const float* __restrict__ q, int off, int nblk, uint32_t stride, int grp,
                                           bool has0, bool has1, float& a0, float& a1)
{
    a0 = 0.f;
    a1 = 0.f;
    for (int c0 = grp; c0 < nblk; c0 += G * kRedUnroll) {
        float x[kRedUnroll], y[kRedUnroll];
#pragma unroll
        for (int k = 0; k < kRedUnroll; ++k) {
            const int c = c0 + G * k;
            x[k] = has0 && c < nblk ? q[(size_t)c * stride] : 0.f;
            y[k] = has1 && c < nblk ? q[(size_t)c * stride + off] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kRedUnroll; ++k) {
            a0 += x[k];
            a1 += y[k];
        }
    }
}

// entry e's total over the block's G groups (group 0's sum first), valid in
// group 0's threads; every thread of the block calls it
template <int G>
__device__ __forceinline__ float block_groups_total(float (*gs)[256 / G], float mine, int q, int e)
{
    if constexpr (G == 1) {
        return mine;
    } else {
        gs[q][e] = mine;
        __syncthreads();
        float a = 0.f;
        if (q == 0)
#pragma unroll
            for (int k = 0; k < G; ++k) a += gs[k][e];
        return a;
    }
}

// The flows' gradients and loss sums from the CTAs' partials, in the fixed
// tree above: grad[f][p] (p < np), then the two loss sums, for the entries
// from p_first on (np: the loss sums alone). A flow without rows gets zeros
// (its CTAs returned before writing). drawn: the gradient was over `batch`
// drawn rows per flow, else over all of each flow's points.
template <int G>
__global__ void __launch_bounds__(256) grad_reduce_kernel(const float* __restrict__ part, int nblk,
                                                          uint32_t part_stride, int np, int p_first,
                                                          const TrainSlot* __restrict__ slots,
                                                          int drawn, uint32_t batch, float* __restrict__ grad,
                                                          float* __restrict__ sums)
{
    constexpr int E = 256 / G;
    __shared__ float gs[G][E];
    const int f = blockIdx.y, e = threadIdx.x % E, q = threadIdx.x / E;
    const int p = p_first + blockIdx.x * E + e;
    const uint64_t n_rows = drawn ? (slots[f].n ? batch : 0) : slots[f].n;
    const float mine =
        n_rows && p < np + 2 ? group_sum<G>(part + (size_t)f * nblk * part_stride + p, nblk, part_stride, q) : 0.f;
    const float a = block_groups_total<G>(gs, mine, q, e);
    if (q != 0 || p >= np + 2) return;
    if (p < np)
        grad[(size_t)f * np + p] = a;
    else
        sums[2 * f + (p - np)] = a;
}


// One Adam update (Kingma, Ba 2015) of a parameter with gradient gr at step
// t >= 1; the fused multiply-adds are written out, so both Adam kernels round
// alike.
// c1 = 1 - b1^t and c2 = 1 - b2^t are the step's bias corrections (adam_bias),
// the same for every parameter.
__device__ __forceinline__ void adam_update(float& param, float& m, float& v, float gr, float c1, float c2, float lr,
                                            float b1, float b2, float eps)
{
    const float mi = __fmaf_rn(b1, m, __fmul_rn(1.f - b1, gr));
    const float vi = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(1.f - b2, gr), gr));
    m = mi;
    v = vi;
    const float mh = __fdiv_rn(mi, c1);
    const float vh = __fdiv_rn(vi, c2);
    param = __fmaf_rn(-lr, __fdiv_rn(mh, __fadd_rn(sqrtf(vh), eps)), param);
}

__device__ __forceinline__ void adam_bias(int t, float b1, float b2, float& c1, float& c2)
{
    c1 = 1.f - powf(b1, (float)t);
    c2 = 1.f - powf(b2, (float)t);
}

__global__ void tick_kernel(int* step) { *step += 1; }

// Early stopping of a training run, one check on the device (block r = flow
// r): the flow's validation loss sum w nll / sum w from the loss sums; a
// lower one than the best so far becomes the best, with a copy of the flow's
// parameters; after `patience` checks in a row without one, the flow stops
// training (its training slot gets no rows, so later steps leave it as it
// is). flags[0] counts the flows still training after the check, flags[1]
// takes the error word (zeroed by the caller).
struct StopState {
    float best;
    int bad;
};

__global__ void __launch_bounds__(256) early_stop_kernel(const float* __restrict__ sums,
                                                         const TrainSlot* __restrict__ val, StopState* st,
                                                         TrainSlot* tr, const float* __restrict__ params,
                                                         float* __restrict__ best, int64_t n_params, int patience,
                                                         const int* __restrict__ err, int* flags)
{
    __shared__ int keep;
    const int r = blockIdx.x;
    if (threadIdx.x == 0) {
        keep = 0;
        const float w = sums[2 * r + 1];
        if (val[r].n > 0 && !(w <= 0.f)) {
            const float vl = __fdiv_rn(sums[2 * r], w);
            StopState s = st[r];
            if (vl < s.best) {
                s.best = vl;
                s.bad = 0;
                keep = 1;
            } else if (++s.bad >= patience && tr[r].n > 0) {
                tr[r].n = 0;
            }
            st[r] = s;
        }
        if (tr[r].n > 0) atomicAdd(&flags[0], 1);
        if (r == 0) flags[1] = *err;
    }
    __syncthreads();
    if (keep)
        for (int64_t i = threadIdx.x; i < n_params; i += blockDim.x)
            best[(size_t)r * n_params + i] = params[(size_t)r * n_params + i];
}

// Master parameter r of one block (W1 [H][8], b1 [H], W2 [16][H], b2 [16]),
// value val, written to every place the published layout holds it: the
// forward and backward operands and the sampler's copy, as BF16 halves of
// their words (masked weights as 0) or whole FP32 words. The words of a layout
// hold two parameters each; storing each half separately lets one thread per
// parameter publish without the other. The layout's padding is never written
// here (a full publish zeroes it).
__device__ __forceinline__ void publish_param(uint32_t* __restrict__ pb, int H, const Layout& L, int r, float val)
{
    unsigned short* h16 = reinterpret_cast<unsigned short*>(pb);
    const int cpd = sampler_cpd(H);
    if (r < 8 * H) {
        const int l = r >> 3, j = r & 7;
        const unsigned short bf = mask1(l, j) ? __bfloat16_as_ushort(__float2bfloat16_rn(val)) : (unsigned short)0;
        const int t = j >> 1;
        // w1: word ((s 8 + g) 4 + t) 2 + h for hidden l = 16 s + g + 8 h
        h16[2 * (L.w1 + (((l >> 4) * 8 + (l & 7)) * 4 + t) * 2 + ((l >> 3) & 1)) + (j & 1)] = bf;
        // w1t: word [j][l / 2]
        h16[2 * (L.w1t + j * (H / 2 + 4) + (l >> 1)) + (l & 1)] = bf;
        // sampler copy: unit l sits at position u of chunk sc
        const int i = l / 7, sc = (l % 7) * cpd + (i >> 4), u = i & 15;
        h16[2 * (L.sw1 + ((sc * 8 + (u & 7)) * 4 + t) * 2 + (u >> 3)) + (j & 1)] = bf;
    } else if (r < 9 * H) {
        const int l = r - 8 * H, rem = l & 15;
        // b1: word (s 4 + t) 4 + q for hidden 16 s + 8 (q / 2) + 2 t + q % 2
        pb[L.b1 + ((l >> 4) * 4 + ((rem & 7) >> 1)) * 4 + ((rem >> 3) << 1 | (rem & 1))] = __float_as_uint(val);
        const int i = l / 7, sc = (l % 7) * cpd + (i >> 4), u = i & 15;
        pb[L.sb1 + (sc * 4 + ((u & 7) >> 1)) * 4 + ((u >> 3) << 1 | (u & 1))] = __float_as_uint(val);
    } else if (r < 25 * H) {
        const int o = (r - 9 * H) / H, l = (r - 9 * H) - o * H, rem = l & 15;
        const unsigned short bf = mask2(o, l) ? __bfloat16_as_ushort(__float2bfloat16_rn(val)) : (unsigned short)0;
        // w2: word ((s 8 + g) 4 + t) 4 + q for output g + 8 (q / 2) and hidden
        // 16 s + 8 (q % 2) + 2 t (+1 in the high half)
        h16[2 * (L.w2 + (((l >> 4) * 8 + (o & 7)) * 4 + ((rem & 7) >> 1)) * 4 + ((o >> 3) << 1 | (rem >> 3))) +
            (l & 1)] = bf;
        // w2t: word l 8 + ((o / 2) ^ (l & 4)), output o / 2 * 2 low, +1 high
        h16[2 * (L.w2t + l * 8 + ((o >> 1) ^ (l & 4))) + (o & 1)] = bf;
        const int i = l / 7, sc = (l % 7) * cpd + (i >> 4), u = i & 15;
        h16[2 * (L.sw2 + ((sc * 8 + (o & 7)) * 4 + ((u & 7) >> 1)) * 4 + ((o >> 3) << 1 | (u >> 3))) + (u & 1)] = bf;
    } else {
        const int o = r - 25 * H;
        pb[L.b2 + o] = __float_as_uint(val);
        pb[L.sb2 + o] = __float_as_uint(val);
    }
}

// A training step's Adam and publish in one launch: adam_kernel on the
// gradient kernel's per-CTA partials, added here in the fixed tree of
// group_sum; each updated parameter is published at once (publish_param). A
// block updates ROWS x 256 / G parameters of flow blockIdx.y (launched with
// two rows: a launch of 16 flows fits one wave, and a one-flow launch leaves
// room on the SMs for the next step's gradient CTAs, which start during it);
// a flow without rows this step keeps its parameters, moments and published
// words. The step t is the gradient launch's ticket count over its CTA count
// (grad_kernel): the counter stands at t grad_ctas after the gradient launch
// of step t - 1, so no launch has to advance a step counter. Launched to
// start during the gradient kernel, the kernel reads its partials and the
// ticket only after that kernel has completed, and releases the next step's
// gradient launch only once the whole block has read the ticket.
template <int G, int ROWS>
__global__ void __launch_bounds__(256) adam_publish_kernel(float* __restrict__ params, const float* __restrict__ part,
                                                           int nblk, uint32_t part_stride,
                                                           const TrainSlot* __restrict__ slots, float* __restrict__ m,
                                                           float* __restrict__ v, const unsigned* __restrict__ ticket,
                                                           uint32_t grad_ctas, uint32_t* __restrict__ pub,
                                                           int K, int H, const __grid_constant__ Layout L,
                                                           int64_t n_params, float lr, float b1, float b2, float eps)
{
    static_assert(ROWS == 1 || ROWS == 2, "one or two rows per block");
    constexpr int E = 256 / G;
    __shared__ float gs[ROWS][G][E];
    __shared__ float w_s, c_s[2];
    // launched to start during the gradient kernel: its partials and ticket
    // are read only after it has completed
    griddep_wait();
    const int f = blockIdx.y, e = threadIdx.x % E, q = threadIdx.x / E;
    const int64_t p0 = (int64_t)blockIdx.x * ROWS * E + e;
    const int t_step = (int)(*ticket / grad_ctas);
    if (threadIdx.x == 32) adam_bias(t_step, b1, b2, c_s[0], c_s[1]);
    const bool has_rows = slots[f].n != 0;   // uniform over the block
    const float* base = part + (size_t)f * nblk * part_stride;
    if (threadIdx.x < 32) {
        // the weight sum: lane j adds CTAs j, j + 32, ... (all loads of a
        // chunk in flight); the lanes' sums meet in lane 0 along a fixed
        // butterfly
        float w = 0.f;
        if (has_rows)
            for (int c0 = threadIdx.x; c0 < nblk; c0 += 32 * 8) {
                float x[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int c = c0 + 32 * k;
                    x[k] = c < nblk ? base[(size_t)c * part_stride + n_params + 1] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) w += x[k];
            }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(kFull, w, off);
        if (threadIdx.x == 0) w_s = w;
    }
    // the parameters and moments this thread updates, loaded with the
    // partials (one round trip for both)
    float pi[ROWS], mi[ROWS], vi[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int64_t p = p0 + r * E, i = (int64_t)f * n_params + p;
        const bool mine = has_rows && q == 0 && p < n_params;
        pi[r] = mine ? params[i] : 0.f;
        mi[r] = mine ? m[i] : 0.f;
        vi[r] = mine ? v[i] : 0.f;
    }
    float g[ROWS];
    if constexpr (ROWS == 1) {
        const float mine = has_rows && p0 < n_params ? group_sum<G>(base + p0, nblk, part_stride, q) : 0.f;
        g[0] = block_groups_total<G>(gs[0], mine, q, e);
    } else {
        float mine0, mine1;
        group_sum2<G>(base + p0, E, nblk, part_stride, q, has_rows && p0 < n_params, has_rows && p0 + E < n_params,
                      mine0, mine1);
        g[0] = block_groups_total<G>(gs[0], mine0, q, e);
        g[1] = block_groups_total<G>(gs[1], mine1, q, e);
    }
    __syncthreads();
    // the block has read the ticket (its bias corrections are in c_s): the
    // next step's gradient kernel may launch and take its tickets
    griddep_release();
    const float W = w_s;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int64_t p = p0 + r * E;
        if (has_rows && q == 0 && p < n_params && W > 0.f) {
            const int64_t i = (int64_t)f * n_params + p;
            adam_update(pi[r], mi[r], vi[r], __fdiv_rn(g[r], W), c_s[0], c_s[1], lr, b1, b2, eps);
            params[i] = pi[r];
            m[i] = mi[r];
            v[i] = vi[r];
            const int mb = master_block(H), b = (int)(p / mb);
            publish_param(pub + ((size_t)f * K + b) * L.words, H, L, (int)(p - (int64_t)b * mb), pi[r]);
        }
    }
}

// n_params per flow; flows one after another. A flow whose weight sum is 0
// (no points this step) keeps its parameters and moments.
__global__ void adam_kernel(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ sums, const int* __restrict__ step,
                            int64_t n_params, int64_t n, float lr, float b1, float b2, float eps)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float W = sums[2 * (i / n_params) + 1];
    if (!(W > 0.f)) return;
    float pi = params[i], mi = m[i], vi = v[i];
    float c1, c2;
    adam_bias(*step, b1, b2, c1, c2);
    adam_update(pi, mi, vi, __fdiv_rn(grad[i], W), c1, c2, lr, b1, b2, eps);
    params[i] = pi;
    m[i] = mi;
    v[i] = vi;
}

}  // namespace maf
}  // namespace abcgb

using namespace abcgb;

struct abc_maf_s {
    int device = 0;
    int R = 1;                 // flows, all with K blocks of H hidden units
    int K = 0, H = 0;
    maf::Box box{};
    int64_t n_params = 0;      // per flow
    int pub_words = 0;         // per block
    float tau = 1.f;           // base scale of sampling and density (training fits tau = 1)
    float* d_params = nullptr; // [R][n_params] FP32 master parameters
    float* d_m = nullptr;
    float* d_v = nullptr;
    float* d_grad = nullptr;
    float* d_part = nullptr;   // [R][CTAs][part_stride] the gradient kernel's per-CTA partials
    size_t part_floats = 0;    // allocated size of d_part
    uint32_t* d_pub = nullptr; // [R][K][pub_words] published BF16 operands
    float* d_sums = nullptr;   // [R][2] (weighted loss sum, weight sum)
    int* d_err = nullptr;      // set by a gradient kernel whose bounded wait ran out
    int hold = 0;              // testing: the gradient kernel issues no products
    int* d_step = nullptr;     // [0] the step of abc_maf_adam_step, [1] a training run's ticket counter
    maf::TrainSlot* d_slots = nullptr;   // [R] training data of each flow
    maf::TrainSlot* d_slots_val = nullptr;   // [R] validation data of each flow (early stopping)
    float* h_io = nullptr;   // pinned host: 2 R floats, then the early-stopping flags [2][2] (int)
    float* d_best = nullptr;   // [R][n_params] best parameters under validation (allocated on first use)
    void* d_stop = nullptr;    // early stopping: [R] StopState, then two pairs of flags (allocated on first use)
    cudaGraphExec_t graph = nullptr;        // one training step, captured
    cudaGraphExec_t graph_multi = nullptr;  // kGraphSteps training steps, captured together
    // what the captured training step was built for
    int32_t g_batch = 0;
    float g_lr = 0.f;
    uint64_t g_seed = 0;
    cudaStream_t g_stream = nullptr;
};

namespace {

#define MAF_TRY(expr, what)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return plan_cuda_fail(_e, what); \
    } while (0)

// After the stream has been synchronised: ABC_ERR_TIMEOUT if a gradient
// kernel's bounded wait for its tensor-core products ran out (the word is
// then cleared for the next call).
abc_status take_err(abc_maf f)
{
    int h = 0;
    MAF_TRY(cudaMemcpy(&h, f->d_err, sizeof h, cudaMemcpyDeviceToHost), "cudaMemcpy(error word)");
    if (h) {
        MAF_TRY(cudaMemset(f->d_err, 0, sizeof h), "cudaMemset(error word)");
        return plan_fail(ABC_ERR_TIMEOUT, "a flow gradient kernel's wait for its tensor-core products ran out of time");
    }
    return ABC_OK;
}

size_t fwd_smem(const abc_maf_s* f) { return sizeof(uint32_t) * (size_t)f->K * maf::layout(f->H).fwd_words; }
size_t samp_smem(const abc_maf_s* f) { return sizeof(uint32_t) * (size_t)f->K * maf::layout(f->H).samp_words; }

size_t grad_smem(const abc_maf_s* f, int warps)
{
    return sizeof(uint32_t) * (size_t)f->K * maf::layout(f->H).grad_words + (size_t)maf::kTcSlot * warps;
}

abc_status check(abc_maf f)
{
    if (!f) return plan_fail(ABC_ERR_INVALID_ARG, "flow is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != f->device)
        return plan_fail(ABC_ERR_INVALID_ARG, "the flow's device is not the current device");
    return ABC_OK;
}

abc_status check_flow(abc_maf f, int32_t r)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (r < 0 || r >= f->R) return plan_fail(ABC_ERR_INVALID_ARG, "flow index out of range");
    return ABC_OK;
}

size_t max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// blocks to launch: all that fit on the GPU at once, or fewer if the work is smaller
template <typename Kern>
int fill_grid(Kern k, int threads, size_t smem, uint64_t want)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const uint64_t cap = (uint64_t)sm_count() * per_sm;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}


// The kernel's dynamic shared-memory limit (one value per kernel and device)
// is only ever raised, so flows of different sizes used from several host
// threads never lower it under a launch that needs more.
template <typename Kern>
cudaError_t allow_smem(Kern k, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& lim = limit[std::make_pair((const void*)k, dev)];
    if (lim >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) lim = bytes;
    return e;
}

const uint32_t* flow_pub(abc_maf f, int r) { return f->d_pub + (size_t)r * f->K * f->pub_words; }

cudaError_t publish(abc_maf f, cudaStream_t s)
{
    const int n = f->K * f->pub_words;
    maf::publish_kernel<<<dim3((n + 255) / 256, f->R), 256, 0, s>>>(f->d_params, f->d_pub, f->K, f->H);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_logq(abc_maf f, int r, uint64_t n, const float* theta, float* logq, cudaStream_t s)
{
    const size_t smem = fwd_smem(f);
    cudaError_t e = allow_smem(maf::logq_kernel<K>, smem);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = (n + 15) / 16;
    const int grid = fill_grid(maf::logq_kernel<K>, maf::kFwdThreads, smem, (tiles + 7) / 8);
    maf::logq_kernel<K><<<grid, maf::kFwdThreads, smem, s>>>(flow_pub(f, r), f->H, f->box, theta, n, 1.f / f->tau, logf(f->tau),
                                                logq);
    return cudaGetLastError();
}

template <int K, int CPD>
cudaError_t launch_sample_c(abc_maf f, int r, uint64_t n, const float* u, const ModelParams& p, uint32_t ctr3,
                            uint64_t first, float* theta, float* logq, cudaStream_t s)
{
    const size_t smem = samp_smem(f);
    cudaError_t e = allow_smem(maf::sample_kernel<K, CPD>, smem);
    if (e != cudaSuccess) return e;
    const uint64_t tiles = (n + 15) / 16;
    const int grid = fill_grid(maf::sample_kernel<K, CPD>, maf::kFwdThreads, smem, (tiles + 7) / 8);
    maf::sample_kernel<K, CPD><<<grid, maf::kFwdThreads, smem, s>>>(flow_pub(f, r), f->H, f->box, u, p, ctr3, first, n, f->tau,
                                                  logf(f->tau), theta, logq);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_sample(abc_maf f, int r, uint64_t n, const float* u, const ModelParams& p, uint32_t ctr3,
                          uint64_t first, float* theta, float* logq, cudaStream_t s)
{
    switch (maf::sampler_cpd(f->H)) {
    case 1: return launch_sample_c<K, 1>(f, r, n, u, p, ctr3, first, theta, logq, s);
    case 2: return launch_sample_c<K, 2>(f, r, n, u, p, ctr3, first, theta, logq, s);
    case 3: return launch_sample_c<K, 3>(f, r, n, u, p, ctr3, first, theta, logq, s);
    default: return cudaErrorInvalidValue;
    }
}

// floats per CTA partial: K blocks of parameters and the two loss sums, padded to 16 bytes
uint32_t part_stride(const abc_maf_s* f) { return (uint32_t)((f->K * maf::master_block(f->H) + 2 + 3) & ~3); }

// The CTA form of a gradient over `tiles` 16-row tiles per flow: compute
// warps per CTA, whether they work in pairs (one tile per pair, each member
// one 128-unit half: half the dependent chain per tile, twice the CTAs), and
// CTAs per flow. The 15-warp form when 4-warp CTAs would run more than two
// waves and it fits; the 4-warp form pairs its warps when the hidden layer has
// two halves.
struct GradForm {
    int W;
    bool pair;
    int grid;
};

int grad_grid(uint64_t tiles, int tiles_per_cta)
{
    const uint64_t want = (tiles + tiles_per_cta - 1) / tiles_per_cta;
    return (int)(want < (uint64_t)sm_count() ? (want > 0 ? want : 1) : (uint64_t)sm_count());
}

GradForm grad_form(abc_maf f, uint64_t tiles)
{
    const uint64_t narrow_ctas = (tiles + maf::kGradWarpsNarrow - 1) / maf::kGradWarpsNarrow * (uint64_t)f->R;
    // the wide form's dynamic shared memory, with 5 KB left for its static part
    GradForm g;
    g.W = (narrow_ctas > 2 * (uint64_t)sm_count() && grad_smem(f, maf::kGradWarpsWide) + 5120 <= max_smem_optin())
              ? maf::kGradWarpsWide
              : maf::kGradWarpsNarrow;
    g.pair = g.W == maf::kGradWarpsNarrow && (f->H + maf::kTcM - 1) / maf::kTcM == 2;
    g.grid = grad_grid(tiles, g.pair ? g.W / 2 : g.W);
    return g;
}

// training steps per replay of the multi-step graph (the validation interval
// of a training run with early stopping)
constexpr int kGraphSteps = 25;

void drop_graphs(abc_maf_s* f)
{
    if (f->graph) cudaGraphExecDestroy(f->graph);
    if (f->graph_multi) cudaGraphExecDestroy(f->graph_multi);
    f->graph = nullptr;
    f->graph_multi = nullptr;
}

// n captured training steps: whole multi-step replays, then single steps
cudaError_t run_steps(abc_maf f, int32_t n, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    for (; n >= kGraphSteps && e == cudaSuccess; n -= kGraphSteps) e = cudaGraphLaunch(f->graph_multi, s);
    for (; n > 0 && e == cudaSuccess; --n) e = cudaGraphLaunch(f->graph, s);
    return e;
}

// the partial buffer for any gradient over at most `tiles` tiles per flow:
// sized for the paired 4-warp form's CTAs (two tiles each), never fewer than
// the other forms' and growing with the tiles; allocates, so it is called
// before a training step is captured
cudaError_t ensure_part(abc_maf f, uint64_t tiles)
{
    const uint64_t grid = (uint64_t)grad_grid(tiles, maf::kGradWarpsNarrow / 2);
    const size_t need = (size_t)f->R * grid * part_stride(f);
    if (need <= f->part_floats) return cudaSuccess;
    // a captured training step holds the old buffer's address
    drop_graphs(f);
    cudaFree(f->d_part);
    f->d_part = nullptr;
    f->part_floats = 0;
    cudaError_t e = cudaMalloc(&f->d_part, sizeof(float) * need);
    if (e == cudaSuccess) f->part_floats = need;
    return e;
}

// groups per entry of the partial reductions over nblk CTAs: the smallest of
// 1, 2, 4, 8 leaving at most kRedUnroll partials per thread
int red_groups(int nblk)
{
    int g = 1;
    while (g < 8 && nblk > g * maf::kRedUnroll) g *= 2;
    return g;
}

template <int G>
void launch_reduce(abc_maf f, const maf::TrainSlot* slots, bool drawn, uint32_t batch, int nblk, uint32_t stride,
                   bool sums_only, cudaStream_t s)
{
    const int np = (int)f->n_params, p_first = sums_only ? np : 0;
    maf::grad_reduce_kernel<G><<<dim3((np + 2 - p_first + 256 / G - 1) / (256 / G), f->R), 256, 0, s>>>(
        f->d_part, nblk, stride, np, p_first, slots, drawn ? 1 : 0, batch, f->d_grad, f->d_sums);
}

// a training run's ticket counter (grad_kernel), zeroed when the run starts
unsigned* train_ticket(abc_maf f) { return reinterpret_cast<unsigned*>(f->d_step + 1); }

template <int G>
cudaError_t launch_adam_publish(abc_maf f, int nblk, float lr, cudaStream_t s)
{
    constexpr int ROWS = 2, PER = ROWS * (256 / G);
    return launch_overlapped(maf::adam_publish_kernel<G, ROWS>, dim3((unsigned)((f->n_params + PER - 1) / PER), f->R),
                             dim3(256), 0, s, f->d_params, f->d_part, nblk, part_stride(f), f->d_slots, f->d_m, f->d_v,
                             train_ticket(f), (uint32_t)nblk * (uint32_t)f->R, f->d_pub, f->K, f->H,
                             maf::layout(f->H), f->n_params, lr, 0.9f, 0.999f, 1e-8f);
}

// gradients of every flow's slot: with a ticket counter, `batch` rows per flow
// drawn for the training step with rp's Philox key; else all max_n points (the
// largest slot). The kernel writes per-CTA partials, the reduction adds them
// in a fixed tree into d_grad and d_sums.
template <int K, int W, bool PAIR>
cudaError_t launch_grad_w(abc_maf f, const maf::TrainSlot* slots, unsigned* ticket, const ModelParams& rp,
                          uint32_t batch, int grid, bool reduce, bool sums_only, cudaStream_t s)
{
    const size_t smem = grad_smem(f, W);
    cudaError_t e = allow_smem(maf::grad_kernel<K, W, PAIR>, smem);
    if (e != cudaSuccess) return e;
    const uint32_t stride = part_stride(f);
    if ((size_t)f->R * grid * stride > f->part_floats) return cudaErrorInvalidValue;   // ensure_part first
    if (PAIR && (f->H + maf::kTcM - 1) / maf::kTcM != 2) return cudaErrorInvalidValue;
    if (ticket)   // a training step: may start while the previous step's Adam finishes
        e = launch_overlapped(maf::grad_kernel<K, W, PAIR>, dim3(grid, f->R), dim3((W + 1) * 32), smem, s, f->d_pub,
                              f->H, f->box, slots, ticket, (uint32_t)grid * (uint32_t)f->R, rp, batch, f->d_part,
                              stride, f->d_err, f->hold);
    else
        maf::grad_kernel<K, W, PAIR><<<dim3(grid, f->R), (W + 1) * 32, smem, s>>>(
            f->d_pub, f->H, f->box, slots, ticket, (uint32_t)grid * (uint32_t)f->R, rp, batch, f->d_part, stride,
            f->d_err, f->hold);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess || !reduce) return e;
    switch (red_groups(grid)) {
    case 1: launch_reduce<1>(f, slots, ticket != nullptr, batch, grid, stride, sums_only, s); break;
    case 2: launch_reduce<2>(f, slots, ticket != nullptr, batch, grid, stride, sums_only, s); break;
    case 4: launch_reduce<4>(f, slots, ticket != nullptr, batch, grid, stride, sums_only, s); break;
    default: launch_reduce<8>(f, slots, ticket != nullptr, batch, grid, stride, sums_only, s); break;
    }
    return cudaGetLastError();
}

// reduce: add the partials into d_grad and d_sums (a training step's Adam adds
// them itself instead)
template <int K>
cudaError_t launch_grad(abc_maf f, const maf::TrainSlot* slots, unsigned* ticket, const ModelParams& rp, uint32_t batch,
                        uint64_t max_n, bool reduce, bool sums_only, cudaStream_t s)
{
    const uint64_t tiles = ((ticket ? batch : max_n) + 15) / 16;
    const GradForm g = grad_form(f, tiles);
    if (g.W == maf::kGradWarpsWide)
        return launch_grad_w<K, maf::kGradWarpsWide, false>(f, slots, ticket, rp, batch, g.grid, reduce, sums_only, s);
    if (g.pair) return launch_grad_w<K, maf::kGradWarpsNarrow, true>(f, slots, ticket, rp, batch, g.grid, reduce, sums_only, s);
    return launch_grad_w<K, maf::kGradWarpsNarrow, false>(f, slots, ticket, rp, batch, g.grid, reduce, sums_only, s);
}

#define MAF_DISPATCH(fn, ...)                      \
    (f->K == 1 ? fn<1>(__VA_ARGS__)                \
     : f->K == 2 ? fn<2>(__VA_ARGS__)              \
     : f->K == 3 ? fn<3>(__VA_ARGS__)              \
                 : fn<4>(__VA_ARGS__))

// the slot table: theta[r], w[r], n[r] for every flow (n[r] = 0: no data).
// The copy is from pageable memory, which the runtime has consumed when the
// call returns, so tables can be uploaded back to back without a wait.
cudaError_t upload_slots(abc_maf f, const float* const* theta, const float* const* w, const uint64_t* n,
                         cudaStream_t s, maf::TrainSlot* dst = nullptr)
{
    std::vector<maf::TrainSlot> h((size_t)f->R);
    for (int r = 0; r < f->R; ++r) {
        h[r].theta = n[r] ? theta[r] : nullptr;
        h[r].w = n[r] && w ? w[r] : nullptr;
        h[r].n = n[r];
    }
    return cudaMemcpyAsync(dst ? dst : f->d_slots, h.data(), sizeof(maf::TrainSlot) * f->R, cudaMemcpyHostToDevice,
                           s);
}

// full-data gradients of the flows described by the slot table
// full-data gradients (sums_only: the loss sums alone reduced, d_grad left as
// it was)
cudaError_t full_gradient(abc_maf f, uint64_t max_n, cudaStream_t s, const maf::TrainSlot* slots = nullptr,
                          bool sums_only = false)
{
    cudaError_t e = ensure_part(f, (max_n + 15) / 16);
    if (e == cudaSuccess)
        e = MAF_DISPATCH(launch_grad, f, slots ? slots : f->d_slots, nullptr, ModelParams{}, 0u, max_n, true, sums_only,
                         s);
    return e;
}

cudaError_t launch_adam(abc_maf f, float lr, float b1, float b2, float eps, cudaStream_t s)
{
    const int64_t n = f->n_params * f->R;
    maf::adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f->d_params, f->d_grad, f->d_m, f->d_v, f->d_sums,
                                                                 f->d_step, f->n_params, n, lr, b1, b2, eps);
    return cudaGetLastError();
}

// one training step on `batch` drawn rows per flow, two launches (captured
// once and replayed): the gradient kernel draws its rows for the current step
// and writes per-CTA partials; Adam adds the partials in a fixed order and
// publishes every updated parameter. Both launches are overlapped
// (programmatic dependent launch): each starts while the previous kernel
// finishes and waits for it before touching its results.
cudaError_t launch_train_step(abc_maf f, uint32_t batch, const ModelParams& p, float lr, cudaStream_t s)
{
    cudaError_t e = MAF_DISPATCH(launch_grad, f, f->d_slots, train_ticket(f), p, batch, 0, false, false, s);
    if (e != cudaSuccess) return e;
    const int grid = grad_form(f, ((uint64_t)batch + 15) / 16).grid;
    switch (red_groups(grid)) {
    case 1: e = launch_adam_publish<1>(f, grid, lr, s); break;
    case 2: e = launch_adam_publish<2>(f, grid, lr, s); break;
    case 4: e = launch_adam_publish<4>(f, grid, lr, s); break;
    default: e = launch_adam_publish<8>(f, grid, lr, s); break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

extern "C" {

abc_status abc_maf_create_multi(int32_t n_flows, int32_t n_blocks, int32_t hidden, const abc_prior_box* box,
                                abc_maf* maf_out)
{
    abc_status st;
    if (!maf_out) return plan_fail(ABC_ERR_INVALID_ARG, "maf_out is NULL");
    *maf_out = nullptr;
    if (!plan_check_prior(box, &st)) return st;
    if (n_flows < 1 || n_flows > ABC_MAF_MAX_FLOWS) return plan_fail(ABC_ERR_INVALID_ARG, "n_flows must be in 1..64");
    if (n_blocks < 1 || n_blocks > maf::kKMax) return plan_fail(ABC_ERR_INVALID_ARG, "n_blocks must be in 1..4");
    if (hidden < 16 || hidden > maf::kHMax || hidden % 16)
        return plan_fail(ABC_ERR_INVALID_ARG, "hidden must be a multiple of 16 in 16..256");
    for (int j = 0; j < 8; ++j)
        if (!(box->hi[j] > box->lo[j])) return plan_fail(ABC_ERR_INVALID_ARG, "the flow needs lo < hi in every coordinate");
    abc_maf_s* f = new abc_maf_s();
    f->R = n_flows;
    f->K = n_blocks;
    f->H = hidden;
    for (int j = 0; j < 8; ++j) {
        f->box.lo[j] = box->lo[j];
        f->box.w[j] = box->hi[j] - box->lo[j];
        f->box.logw[j] = logf(f->box.w[j]);
    }
    f->n_params = (int64_t)n_blocks * maf::master_block(hidden);
    f->pub_words = maf::layout(hidden).words;
    auto fail_free = [f](abc_status e) {
        abc_maf_destroy(f);
        return e;
    };
    if (grad_smem(f, maf::kGradWarpsNarrow) > max_smem_optin())
        return fail_free(plan_fail(ABC_ERR_INVALID_ARG,
                                   "the gradient kernel of this flow (blocks x hidden) needs more shared memory per "
                                   "block than the device has; use fewer blocks or hidden units"));
    const size_t np = sizeof(float) * f->n_params * f->R;
    cudaError_t e;
    if ((e = cudaGetDevice(&f->device)) != cudaSuccess || (e = cudaMalloc(&f->d_params, np)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_m, np)) != cudaSuccess || (e = cudaMalloc(&f->d_v, np)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_grad, np)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_pub, sizeof(uint32_t) * (size_t)f->R * f->K * f->pub_words)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_sums, 2 * sizeof(float) * f->R)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_step, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&f->d_slots, sizeof(maf::TrainSlot) * f->R)) != cudaSuccess ||
        (e = cudaMalloc(&f->d_slots_val, sizeof(maf::TrainSlot) * f->R)) != cudaSuccess ||
        (e = cudaMallocHost(&f->h_io, sizeof(float) * (2 * (size_t)f->R + 4))) != cudaSuccess ||
        (e = cudaMalloc(&f->d_err, sizeof(int))) != cudaSuccess)
        return fail_free(plan_cuda_fail(e, "cudaMalloc(flow)"));
    if ((e = cudaMemset(f->d_params, 0, np)) != cudaSuccess || (e = cudaMemset(f->d_m, 0, np)) != cudaSuccess ||
        (e = cudaMemset(f->d_v, 0, np)) != cudaSuccess || (e = cudaMemset(f->d_step, 0, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(f->d_slots, 0, sizeof(maf::TrainSlot) * f->R)) != cudaSuccess ||
        (e = cudaMemset(f->d_err, 0, sizeof(int))) != cudaSuccess ||
        (e = publish(f, nullptr)) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess)
        return fail_free(plan_cuda_fail(e, "flow initialisation"));
    *maf_out = f;
    return plan_ok();
}

abc_status abc_maf_create(int32_t n_blocks, int32_t hidden, const abc_prior_box* box, abc_maf* maf_out)
{
    return abc_maf_create_multi(1, n_blocks, hidden, box, maf_out);
}

int64_t abc_maf_param_count(abc_maf f) { return f ? f->n_params : -1; }

int32_t abc_maf_flow_count(abc_maf f) { return f ? f->R : -1; }

abc_status abc_maf_test_hold_products(abc_maf f, int32_t hold)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    f->hold = hold != 0;
    drop_graphs(f);
    return plan_ok();
}

abc_status abc_maf_set_proposal_scale(abc_maf f, float tau)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (!(tau >= 0.5f && tau <= 4.f)) return plan_fail(ABC_ERR_INVALID_ARG, "tau must be in [0.5, 4]");
    f->tau = tau;
    return plan_ok();
}

abc_status abc_maf_init_random(abc_maf f, uint64_t seed, float scale)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (!(scale >= 0.f)) return plan_fail(ABC_ERR_INVALID_ARG, "scale must be >= 0");
    std::vector<float> v((size_t)f->n_params * f->R, 0.f);
    std::mt19937_64 gen(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    const int H = f->H, mb = maf::master_block(H);
    for (int b = 0; b < f->K * f->R; ++b) {
        float* M = v.data() + (size_t)b * mb;
        for (int i = 0; i < 8 * H; ++i) M[i] = nd(gen) * scale / sqrtf(8.f);
        for (int i = 0; i < 16 * H; ++i) M[9 * H + i] = nd(gen) * scale / sqrtf((float)H);
    }
    return abc_maf_set_params(f, v.data());
}

abc_status abc_maf_set_params(abc_maf f, const float* params)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (!params) return plan_fail(ABC_ERR_INVALID_ARG, "params is NULL");
    const size_t np = sizeof(float) * f->n_params * f->R;
    MAF_TRY(cudaMemcpy(f->d_params, params, np, cudaMemcpyHostToDevice), "cudaMemcpy(params)");
    MAF_TRY(cudaMemset(f->d_m, 0, np), "cudaMemset");
    MAF_TRY(cudaMemset(f->d_v, 0, np), "cudaMemset");
    MAF_TRY(cudaMemset(f->d_step, 0, 2 * sizeof(int)), "cudaMemset");
    MAF_TRY(publish(f, nullptr), "publish");
    MAF_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return plan_ok();
}

abc_status abc_maf_get_params(abc_maf f, float* params)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (!params) return plan_fail(ABC_ERR_INVALID_ARG, "params is NULL");
    MAF_TRY(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    MAF_TRY(cudaMemcpy(params, f->d_params, sizeof(float) * f->n_params * f->R, cudaMemcpyDeviceToHost),
            "cudaMemcpy(params)");
    return plan_ok();
}

abc_status abc_maf_sample_at(abc_maf f, int32_t flow, uint64_t n, const float* base_draws, uint64_t seed,
                             uint32_t stream, uint64_t first_index, float* theta_out, float* logq_out,
                             void* cuda_stream)
{
    abc_status st;
    if ((st = check_flow(f, flow)) != ABC_OK) return st;
    if (n && !theta_out) return plan_fail(ABC_ERR_INVALID_ARG, "theta_out is NULL");
    if (stream > ABC_STREAM_MAX) return plan_fail(ABC_ERR_INVALID_ARG, "stream above 2^30 - 1");
    if (n == 0) return plan_ok();
    const ModelParams p = plan_make_params(nullptr, 1, 1, seed, stream, nullptr);
    MAF_TRY(MAF_DISPATCH(launch_sample, f, flow, n, base_draws, p, stream << 2, first_index, theta_out, logq_out,
                         (cudaStream_t)cuda_stream),
            "flow sample launch");
    return plan_ok();
}

abc_status abc_maf_sample(abc_maf f, uint64_t n, const float* base_draws, uint64_t seed, uint32_t stream,
                          uint64_t first_index, float* theta_out, float* logq_out, void* cuda_stream)
{
    return abc_maf_sample_at(f, 0, n, base_draws, seed, stream, first_index, theta_out, logq_out, cuda_stream);
}

abc_status abc_maf_log_q_at(abc_maf f, int32_t flow, uint64_t n, const float* theta, float* logq_out,
                            void* cuda_stream)
{
    abc_status st;
    if ((st = check_flow(f, flow)) != ABC_OK) return st;
    if (n && (!theta || !logq_out)) return plan_fail(ABC_ERR_INVALID_ARG, "NULL device buffer");
    if (n == 0) return plan_ok();
    MAF_TRY(MAF_DISPATCH(launch_logq, f, flow, n, theta, logq_out, (cudaStream_t)cuda_stream), "flow log_q launch");
    return plan_ok();
}

abc_status abc_maf_log_q(abc_maf f, uint64_t n, const float* theta, float* logq_out, void* cuda_stream)
{
    return abc_maf_log_q_at(f, 0, n, theta, logq_out, cuda_stream);
}

abc_status abc_maf_gradient(abc_maf f, uint64_t n, const float* theta, const float* weights, float* loss_out,
                            float* grads_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (n == 0 || !theta) return plan_fail(ABC_ERR_INVALID_ARG, "need n > 0 points");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // flow 0 only: the other flows get no points
    std::vector<const float*> th((size_t)f->R, nullptr), w((size_t)f->R, nullptr);
    std::vector<uint64_t> nn((size_t)f->R, 0);
    th[0] = theta;
    w[0] = weights;
    nn[0] = n;
    MAF_TRY(upload_slots(f, th.data(), w.data(), nn.data(), s), "cudaMemcpyAsync(slots)");
    MAF_TRY(full_gradient(f, n, s), "flow gradient");
    float sums[2] = {0.f, 0.f};
    MAF_TRY(cudaMemcpyAsync(sums, f->d_sums, sizeof sums, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(sums)");
    MAF_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    {
        const abc_status es = take_err(f);
        if (es != ABC_OK) return es;
    }
    if (loss_out) *loss_out = sums[1] > 0.f ? sums[0] / sums[1] : 0.f;
    if (grads_out) {
        MAF_TRY(cudaMemcpy(grads_out, f->d_grad, sizeof(float) * f->n_params, cudaMemcpyDeviceToHost),
                "cudaMemcpy(grad)");
        const float W = sums[1] > 0.f ? sums[1] : 1.f;
        for (int64_t i = 0; i < f->n_params; ++i) grads_out[i] /= W;
    }
    return plan_ok();
}

abc_status abc_maf_adam_step(abc_maf f, float lr, float beta1, float beta2, float eps, void* cuda_stream)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    maf::tick_kernel<<<1, 1, 0, s>>>(f->d_step);
    MAF_TRY(launch_adam(f, lr, beta1, beta2, eps, s), "adam launch");
    MAF_TRY(publish(f, s), "publish");
    return plan_ok();
}

abc_status abc_maf_train_flows(abc_maf f, const float* const* theta, const float* const* weights, const uint64_t* n,
                               int32_t n_steps, int32_t batch, float lr, uint64_t seed, float val_fraction,
                               float* loss_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (!theta || !n || n_steps < 0 || batch < 16)
        return plan_fail(ABC_ERR_INVALID_ARG, "need theta and n tables, n_steps >= 0 and batch >= 16");
    if (!(val_fraction >= 0.f) || val_fraction > 0.5f)
        return plan_fail(ABC_ERR_INVALID_ARG, "val_fraction must be in [0, 0.5]");
    uint64_t max_n = 0;
    for (int r = 0; r < f->R; ++r) {
        if (n[r] && !theta[r]) return plan_fail(ABC_ERR_INVALID_ARG, "a flow with points has theta NULL");
        if (n[r] > 0xFFFFFFFFull) return plan_fail(ABC_ERR_INVALID_ARG, "more than 2^32 - 1 points for one flow");
        max_n = n[r] > max_n ? n[r] : max_n;
    }
    if (max_n == 0) return plan_fail(ABC_ERR_INVALID_ARG, "no flow has points");
    // the last floor(val_fraction n) points of a flow, at most kMaxVal,
    // validate; the rest train
    constexpr uint64_t kMaxVal = 8192;
    const int R = f->R;
    std::vector<const float*> th_tr(theta, theta + R), w_tr((size_t)R, nullptr), th_va((size_t)R, nullptr),
        w_va((size_t)R, nullptr);
    std::vector<uint64_t> n_tr(n, n + R), n_va((size_t)R, 0);
    bool validate = false;
    for (int r = 0; r < R; ++r) {
        w_tr[r] = weights ? weights[r] : nullptr;
        uint64_t v = val_fraction > 0.f && n[r] >= 20 ? (uint64_t)std::floor(val_fraction * (double)n[r]) : 0;
        if (v > kMaxVal) v = kMaxVal;
        if (v > 0) {
            n_va[r] = v;
            n_tr[r] = n[r] - v;
            th_va[r] = theta[r] + 8 * n_tr[r];
            w_va[r] = w_tr[r] ? w_tr[r] + n_tr[r] : nullptr;
            validate = true;
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s && n_steps > 0) return plan_fail(ABC_ERR_INVALID_ARG, "training needs a non-default stream");
    MAF_TRY(upload_slots(f, th_tr.data(), w_tr.data(), n_tr.data(), s), "cudaMemcpyAsync(slots)");
    // the gradient partials for both the training batches and the validation
    // sets, allocated before the step is captured (a later reallocation would
    // drop the captured step)
    {
        uint64_t max_va = 0;
        for (int r = 0; r < R; ++r) max_va = n_va[r] > max_va ? n_va[r] : max_va;
        const uint64_t rows = std::max<uint64_t>((uint64_t)batch, max_va);
        MAF_TRY(ensure_part(f, (rows + 15) / 16), "cudaMalloc(gradient partials)");
    }
    // fresh Adam moments for this training run
    const size_t np = sizeof(float) * f->n_params * f->R;
    MAF_TRY(cudaMemsetAsync(f->d_m, 0, np, s), "cudaMemsetAsync");
    MAF_TRY(cudaMemsetAsync(f->d_v, 0, np, s), "cudaMemsetAsync");
    MAF_TRY(cudaMemsetAsync(f->d_step, 0, 2 * sizeof(int), s), "cudaMemsetAsync");
    if (n_steps > 0) {
        // the step reads its data through the slot table, so a graph captured
        // for (batch, lr, seed, stream) serves every data set
        const bool same = f->graph && f->g_batch == batch && f->g_lr == lr && f->g_seed == seed && f->g_stream == s;
        if (!same) {
            drop_graphs(f);
            const ModelParams p = plan_make_params(nullptr, 1, 1, seed, 0, nullptr);
            // one step, and kGraphSteps steps in one graph (the steps take
            // their step number from the ticket counter, so every replay of
            // either continues where the last one stopped)
            for (int which = 0; which < 2; ++which) {
                cudaGraph_t gph = nullptr;
                MAF_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
                cudaError_t e = cudaSuccess;
                for (int i = 0; i < (which ? kGraphSteps : 1) && e == cudaSuccess; ++i)
                    e = launch_train_step(f, (uint32_t)batch, p, lr, s);
                cudaError_t ec = cudaStreamEndCapture(s, &gph);
                if (e != cudaSuccess || ec != cudaSuccess) {
                    if (gph) cudaGraphDestroy(gph);
                    drop_graphs(f);
                    return plan_cuda_fail(e != cudaSuccess ? e : ec, "capturing the training step");
                }
                e = cudaGraphInstantiate(which ? &f->graph_multi : &f->graph, gph, 0);
                cudaGraphDestroy(gph);
                if (e != cudaSuccess) {
                    drop_graphs(f);
                    return plan_cuda_fail(e, "cudaGraphInstantiate(training step)");
                }
            }
            f->g_batch = batch;
            f->g_lr = lr;
            f->g_seed = seed;
            f->g_stream = s;
        }
    }
    if (validate) {
        // early stopping: every kCheck steps the validation loss of each flow;
        // a flow keeps its best parameters and stops after kPatience checks
        // without improvement
        constexpr int kCheck = kGraphSteps, kPatience = 3;
        const size_t npb = sizeof(float) * f->n_params;
        if (!f->d_best) MAF_TRY(cudaMalloc(&f->d_best, npb * R), "cudaMalloc(best parameters)");
        uint64_t max_va = 0;
        for (int r = 0; r < R; ++r) max_va = n_va[r] > max_va ? n_va[r] : max_va;
        // the validation sets have their own slot table, uploaded once. Each
        // check runs on the device (early_stop_kernel: best loss, the best
        // parameters' copy, a stopped flow's training slot emptied), and the
        // host reads its flags (flows still training, the error word) one
        // check late: the GPU meanwhile runs the next steps and check, and at
        // most one replay of steps runs after every flow has stopped (steps
        // leave a flow without rows as it is).
        MAF_TRY(upload_slots(f, th_va.data(), w_va.data(), n_va.data(), s, f->d_slots_val), "cudaMemcpyAsync(slots)");
        const size_t stop_bytes = sizeof(maf::StopState) * R;
        if (!f->d_stop) MAF_TRY(cudaMalloc(&f->d_stop, stop_bytes + 4 * sizeof(int)), "cudaMalloc(early stopping)");
        maf::StopState* d_st = static_cast<maf::StopState*>(f->d_stop);
        int* d_flags = reinterpret_cast<int*>(static_cast<char*>(f->d_stop) + stop_bytes);   // [2][2]
        {
            const std::vector<maf::StopState> init((size_t)R, maf::StopState{INFINITY, 0});
            MAF_TRY(cudaMemcpyAsync(d_st, init.data(), stop_bytes, cudaMemcpyHostToDevice, s),
                    "cudaMemcpyAsync(early stopping)");
        }
        int* flags_h = reinterpret_cast<int*>(f->h_io + 2 * (size_t)R);   // [2][2] in pinned memory
        struct Events {
            cudaEvent_t e[2] = {nullptr, nullptr};
            ~Events()
            {
                for (cudaEvent_t x : e)
                    if (x) cudaEventDestroy(x);
            }
        } ev;
        for (cudaEvent_t& x : ev.e) MAF_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "cudaEventCreate");
        int checks = 0;
        auto check = [&]() -> abc_status {
            const int slot = checks & 1;
            MAF_TRY(full_gradient(f, max_va, s, f->d_slots_val, true), "validation loss");
            MAF_TRY(cudaMemsetAsync(d_flags + 2 * slot, 0, 2 * sizeof(int), s), "cudaMemsetAsync(flags)");
            maf::early_stop_kernel<<<R, 256, 0, s>>>(f->d_sums, f->d_slots_val, d_st, f->d_slots, f->d_params,
                                                     f->d_best, f->n_params, kPatience, f->d_err, d_flags + 2 * slot);
            MAF_TRY(cudaGetLastError(), "early stopping launch");
            MAF_TRY(cudaMemcpyAsync(flags_h + 2 * slot, d_flags + 2 * slot, 2 * sizeof(int), cudaMemcpyDeviceToHost, s),
                    "cudaMemcpyAsync(flags)");
            MAF_TRY(cudaEventRecord(ev.e[slot], s), "cudaEventRecord");
            ++checks;
            return ABC_OK;
        };
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || n_tr[r] > 0;
        if ((st = check()) != ABC_OK) return st;
        for (int32_t done = 0; any && done < n_steps;) {
            if (checks >= 2) {
                // the check before the last one enqueued
                const int slot = checks & 1;
                MAF_TRY(cudaEventSynchronize(ev.e[slot]), "cudaEventSynchronize");
                if (flags_h[2 * slot + 1]) break;   // a wait ran out: reported below
                if (flags_h[2 * slot] == 0) break;  // every flow has stopped
            }
            const int32_t k = n_steps - done < kCheck ? n_steps - done : kCheck;
            MAF_TRY(run_steps(f, k, s), "cudaGraphLaunch");
            done += k;
            if ((st = check()) != ABC_OK) return st;
        }
        // the kept parameters: each validated flow's best
        for (int r = 0; r < R; ++r)
            if (n_va[r] > 0)
                MAF_TRY(cudaMemcpyAsync(f->d_params + (size_t)r * f->n_params, f->d_best + (size_t)r * f->n_params, npb,
                                        cudaMemcpyDeviceToDevice, s),
                        "cudaMemcpyAsync(restore parameters)");
        MAF_TRY(publish(f, s), "publish");
        std::vector<maf::StopState> fin((size_t)R);
        MAF_TRY(cudaMemcpyAsync(fin.data(), d_st, stop_bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(early stopping)");
        MAF_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        {
            const abc_status es = take_err(f);
            if (es != ABC_OK) return es;
        }
        if (loss_out)
            for (int r = 0; r < R; ++r) loss_out[r] = n_va[r] > 0 && fin[r].best < INFINITY ? fin[r].best : 0.f;
        return plan_ok();
    }
    if (n_steps > 0) {
        // each step publishes every parameter it updates, the sampler's
        // operands included
        MAF_TRY(run_steps(f, n_steps, s), "cudaGraphLaunch");
    }
    if (loss_out) {
        MAF_TRY(full_gradient(f, max_n, s), "flow loss");
        std::vector<float> sums(2 * (size_t)f->R);
        MAF_TRY(cudaMemcpyAsync(sums.data(), f->d_sums, sizeof(float) * sums.size(), cudaMemcpyDeviceToHost, s),
                "cudaMemcpyAsync(sums)");
        MAF_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        {
            const abc_status es = take_err(f);
            if (es != ABC_OK) return es;
        }
        for (int r = 0; r < f->R; ++r) loss_out[r] = sums[2 * r + 1] > 0.f ? sums[2 * r] / sums[2 * r + 1] : 0.f;
    } else {
        MAF_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        {
            const abc_status es = take_err(f);
            if (es != ABC_OK) return es;
        }
    }
    return plan_ok();
}

abc_status abc_maf_train(abc_maf f, uint64_t n, const float* theta, const float* weights, int32_t n_steps,
                         int32_t batch, float lr, uint64_t seed, float* loss_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check(f)) != ABC_OK) return st;
    if (n == 0 || !theta) return plan_fail(ABC_ERR_INVALID_ARG, "need n > 0 points");
    // flow 0 only: the other flows get no points and keep their parameters
    std::vector<const float*> th((size_t)f->R, nullptr), w((size_t)f->R, nullptr);
    std::vector<uint64_t> nn((size_t)f->R, 0);
    std::vector<float> loss((size_t)f->R, 0.f);
    th[0] = theta;
    w[0] = weights;
    nn[0] = n;
    st = abc_maf_train_flows(f, th.data(), w.data(), nn.data(), n_steps, batch, lr, seed, 0.f,
                             loss_out ? loss.data() : nullptr, cuda_stream);
    if (st == ABC_OK && loss_out) *loss_out = loss[0];
    return st;
}

abc_status abc_maf_destroy(abc_maf f)
{
    if (!f) return plan_fail(ABC_ERR_INVALID_ARG, "flow is NULL");
    drop_graphs(f);
    cudaFree(f->d_params);
    cudaFree(f->d_m);
    cudaFree(f->d_v);
    cudaFree(f->d_grad);
    cudaFree(f->d_part);
    cudaFree(f->d_pub);
    cudaFree(f->d_sums);
    cudaFree(f->d_step);
    cudaFree(f->d_slots);
    cudaFree(f->d_slots_val);
    if (f->h_io) cudaFreeHost(f->h_io);
    cudaFree(f->d_err);
    cudaFree(f->d_best);
    cudaFree(f->d_stop);
    delete f;
    // leaves the thread's last error as it was: drivers destroy their flows
    // on the way out of a failed call
    return ABC_OK;
}

}  // extern "C"
