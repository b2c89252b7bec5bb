// abc_smc.cu -- sequential ABC with the learned flow proposal: the host loop
// over rounds (propose, simulate and accept, weight, train, shrink eps).
// Every step runs in the library's kernels: the flow sampler and trainer
// (abc_maf.cu) and the batched rejection kernel of a one-region plan
// (abc_batch.cu) reading the proposals from device memory.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/abc_gb300.h"
#include "abc_model.cuh"

namespace abcgb {
abc_status plan_fail(abc_status st, const char* msg);
abc_status plan_cuda_fail(cudaError_t e, const char* what);
abc_status plan_ok();
bool plan_check_prior(const abc_prior_box* prior, abc_status* st);
ModelParams plan_make_params(const abc_prior_box* prior, int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream,
                             const int32_t* ard0);
abc_status plan_results_all(abc_plan plan, uint64_t* n_accepted, uint64_t* simulated_days, float** theta_out,
                            double** dist_out, uint64_t** idx_out, void* cuda_stream);
}  // namespace abcgb

namespace {

// prior draws of sample indices first .. first + n - 1 (stream 0, the words the
// plain sampler would use for those indices)
__global__ void prior_theta_kernel(const __grid_constant__ abcgb::ModelParams p, uint64_t first, uint64_t n,
                                   float* __restrict__ theta)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float th[8];
    abcgb::prior_draw(p, first + j, th);
    float4* o = reinterpret_cast<float4*>(theta + 8 * j);
    o[0] = make_float4(th[0], th[1], th[2], th[3]);
    o[1] = make_float4(th[4], th[5], th[6], th[7]);
}

// log q_mix = log((1 - lam) q + lam prior), in place over log q
__global__ void mixture_logq_kernel(float* __restrict__ logq, uint64_t n, float log_1m_lam, float log_lam_prior)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float a = log_1m_lam + logq[j], b = log_lam_prior;
    const float m = fmaxf(a, b);
    logq[j] = m + log1pf(expf(-fabsf(a - b)));
}

// Importance weights of a round's m accepted samples, on the device.
// Pass 1: log w_j = log prior - log q_mix(theta_j) (0 for prior draws, logq
// NULL), and the maximum (atomicMax over an order-preserving integer key).
// Pass 2: v_j = exp(log w_j - max) in double; sum v and sum v^2 (for the ESS);
// v_j as the float training weight, optionally v_j in double for every j and
// for the first pool_k samples.
struct WeightScratch {
    unsigned int max_key;
    unsigned int pad;
    double sums[2];
    unsigned long long n_tail;   // accepted samples with index >= tail_first (the defensive prior draws)
};

__device__ __forceinline__ unsigned int float_key(float f)
{
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(unsigned int k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ void logw_body(const float* __restrict__ logq, const uint64_t* __restrict__ idx, uint64_t first, uint64_t m,
                            uint64_t tail_first, float log_prior, float* __restrict__ lw, WeightScratch* ws)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float v = -INFINITY;
    bool tail = false;
    if (j < m) {
        v = logq ? log_prior - logq[idx[j] - first] : 0.f;
        lw[j] = v;
        tail = idx[j] >= tail_first;
    }
    const unsigned int n_tail = __popc(__ballot_sync(0xFFFFFFFFu, tail));
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, off));
    if ((threadIdx.x & 31) == 0) {
        if (v > -INFINITY) atomicMax(&ws->max_key, float_key(v));
        if (n_tail) atomicAdd(&ws->n_tail, (unsigned long long)n_tail);
    }
}

__global__ void logw_kernel(const float* __restrict__ logq, const uint64_t* __restrict__ idx, uint64_t first, uint64_t m,
                            uint64_t tail_first, float log_prior, float* __restrict__ lw, WeightScratch* ws)
{
    logw_body(logq, idx, first, m, tail_first, log_prior, lw, ws);
}

__device__ __forceinline__ void weight_body(const float* __restrict__ lw, uint64_t m, WeightScratch* ws, float* __restrict__ w_train,
                              double* __restrict__ w_exact, double* __restrict__ pool, uint64_t pool_k, double power,
                              double* __restrict__ block_sums)
{
    __shared__ double part[2][8];
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double top = (double)key_float(ws->max_key);
    double v = 0.0;
    if (j < m) {
        const double l = (double)lw[j];
        v = exp(l - top);
        w_train[j] = (float)(power == 1.0 ? v : exp(power * (l - top)));
        if (w_exact) w_exact[j] = v;
        if (pool && j < pool_k) pool[j] = v;
    }
    double a = v, b = v * v;
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xFFFFFFFFu, a, off);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, off);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        part[0][warp] = a;
        part[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            sa += part[0][k];
            sb += part[1][k];
        }
        block_sums[2 * blockIdx.x] = sa;
        block_sums[2 * blockIdx.x + 1] = sb;
    }
}

__global__ void weight_kernel(const float* __restrict__ lw, uint64_t m, WeightScratch* ws, float* __restrict__ w_train,
                              double* __restrict__ w_exact, double* __restrict__ pool, uint64_t pool_k, double power,
                              double* __restrict__ block_sums)
{
    weight_body(lw, m, ws, w_train, w_exact, pool, pool_k, power, block_sums);
}

// sum v and sum v^2 from the blocks' sums (one block of 256): thread t adds
// blocks t, t + 256, ... in turn, then the threads' sums meet in a fixed
// pairwise tree (t += t + 128, then t + 64, ...), so the sums are the same in
// every run. (Thread 0 adding the 256 sums in turn took about 20 us: a chain of
// 512 dependent double additions.)
__device__ __forceinline__ void weight_sums_body(const double* __restrict__ block_sums, unsigned nblk,
                                                          WeightScratch* ws)
{
    __shared__ double part[2][256];
    double a = 0.0, b = 0.0;
    for (unsigned k = threadIdx.x; k < nblk; k += 256) {
        a += block_sums[2 * k];
        b += block_sums[2 * k + 1];
    }
    part[0][threadIdx.x] = a;
    part[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            part[0][threadIdx.x] += part[0][threadIdx.x + w];
            part[1][threadIdx.x] += part[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ws->sums[0] = part[0][0];
        ws->sums[1] = part[1][0];
    }
}

__global__ void __launch_bounds__(256) weight_sums_kernel(const double* __restrict__ block_sums, unsigned nblk,
                                                          WeightScratch* ws)
{
    weight_sums_body(block_sums, nblk, ws);
}

// ---------------------------------------------------------------------------
// The accepted samples of a run in ascending sample index. The batched kernel
// hands out accept slots with atomicAdd, so its buffers' order changes from
// run to run; the drivers build the weights, the pools and the training sets
// from this sorted copy, which makes every later step (training-set split,
// batch rows, hence the trained flows) the same in every run with one seed.
// A run's indices lie in [first, first + n): pos[i - first] takes the accept
// slot of index i (all ones for none), a scan over 1024-index blocks gives
// each accepted index its rank, and the gather writes the samples by rank.
// ---------------------------------------------------------------------------
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;
constexpr int kSortBlock = 1024;   // indices per scan block (256 threads x 4)

__device__ __forceinline__ void scatter_slots_body(const uint64_t* __restrict__ idx, uint64_t m, uint64_t first,
                                     uint32_t* __restrict__ pos)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) pos[idx[j] - first] = (uint32_t)j;
}

__global__ void scatter_slots_kernel(const uint64_t* __restrict__ idx, uint64_t m, uint64_t first,
                                     uint32_t* __restrict__ pos)
{
    scatter_slots_body(idx, m, first, pos);
}

// exclusive scan of the 256 threads' counts; returns this thread's offset, *total the block's sum
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t warp_sums[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < 8; ++w) {
        if (w < warp) before += warp_sums[w];
        all += warp_sums[w];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

__device__ __forceinline__ void count_slots_body(const uint32_t* __restrict__ pos, uint64_t n,
                                                          uint32_t* __restrict__ block_count)
{
    const uint64_t base = (uint64_t)blockIdx.x * kSortBlock + 4 * threadIdx.x;
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) c += (base + q < n && pos[base + q] != kNoSlot) ? 1u : 0u;
    uint32_t total = 0;
    block_exclusive_scan(c, &total);
    if (threadIdx.x == 0) block_count[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) count_slots_kernel(const uint32_t* __restrict__ pos, uint64_t n,
                                                          uint32_t* __restrict__ block_count)
{
    count_slots_body(pos, n, block_count);
}

// in-place exclusive scan of nb block counts, one block of 256 threads, in order
__device__ __forceinline__ void scan_counts_body(uint32_t* __restrict__ count, uint32_t nb)
{
    uint32_t carry = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += 256) {
        const uint32_t b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? count[b] : 0u;
        uint32_t total = 0;
        const uint32_t off = block_exclusive_scan(v, &total);
        if (b < nb) count[b] = carry + off;
        carry += total;
    }
}

__global__ void __launch_bounds__(256) scan_counts_kernel(uint32_t* __restrict__ count, uint32_t nb)
{
    scan_counts_body(count, nb);
}

__device__ __forceinline__ void gather_sorted_body(const uint32_t* __restrict__ pos, uint64_t n,
                                                            const uint32_t* __restrict__ block_off,
                                                            const float* __restrict__ theta,
                                                            const double* __restrict__ dist,
                                                            const uint64_t* __restrict__ idx,
                                                            float* __restrict__ theta_o, double* __restrict__ dist_o,
                                                            uint64_t* __restrict__ idx_o)
{
    const uint64_t base = (uint64_t)blockIdx.x * kSortBlock + 4 * threadIdx.x;
    uint32_t slot[4], c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        slot[q] = base + q < n ? pos[base + q] : kNoSlot;
        c += slot[q] != kNoSlot ? 1u : 0u;
    }
    uint32_t total = 0;
    uint32_t r = block_off[blockIdx.x] + block_exclusive_scan(c, &total);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (slot[q] == kNoSlot) continue;
        const float4* src = reinterpret_cast<const float4*>(theta + 8 * (size_t)slot[q]);
        float4* dst = reinterpret_cast<float4*>(theta_o + 8 * (size_t)r);
        dst[0] = src[0];
        dst[1] = src[1];
        dist_o[r] = dist[slot[q]];
        idx_o[r] = idx[slot[q]];
        ++r;
    }
}

__global__ void __launch_bounds__(256) gather_sorted_kernel(const uint32_t* __restrict__ pos, uint64_t n,
                                                            const uint32_t* __restrict__ block_off,
                                                            const float* __restrict__ theta,
                                                            const double* __restrict__ dist,
                                                            const uint64_t* __restrict__ idx,
                                                            float* __restrict__ theta_o, double* __restrict__ dist_o,
                                                            uint64_t* __restrict__ idx_o)
{
    gather_sorted_body(pos, n, block_off, theta, dist, idx, theta_o, dist_o, idx_o);
}

// training set: dst[j] = src[(a j + b) mod m] for theta and weights, j < n <= m
// (a coprime to m, so a permutation): the held-out tail of the training set is
// then a spread-out subset of the data, not its highest sample indices
template <typename W>
__device__ __forceinline__ void permute_body(const float* __restrict__ theta, const W* __restrict__ w, uint64_t m, uint64_t n,
                               uint64_t a, uint64_t b, float* __restrict__ theta_dst, float* __restrict__ w_dst)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t i = (a * j + b) % m;
    const float4* src = reinterpret_cast<const float4*>(theta + 8 * i);
    float4* dst = reinterpret_cast<float4*>(theta_dst + 8 * j);
    dst[0] = src[0];
    dst[1] = src[1];
    w_dst[j] = (float)w[i];
}

template <typename W>
__global__ void permute_kernel(const float* __restrict__ theta, const W* __restrict__ w, uint64_t m, uint64_t n,
                               uint64_t a, uint64_t b, float* __restrict__ theta_dst, float* __restrict__ w_dst)
{
    permute_body<W>(theta, w, m, n, a, b, theta_dst, w_dst);
}

__device__ __forceinline__ void scale_body(double* __restrict__ w, uint64_t m, double f)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) w[j] *= f;
}

__global__ void scale_kernel(double* __restrict__ w, uint64_t m, double f)
{
    scale_body(w, m, f);
}

// ---------------------------------------------------------------------------
// A round's results of many regions in one launch per step (grid row y =
// region): the steps above, each region on its own slice of per-region
// scratch. A block past its region's size returns at once.
// ---------------------------------------------------------------------------
struct RegionRound {
    const float* acc_theta;    // the plan's accepted samples (accept-slot order)
    const double* acc_dist;
    const uint64_t* acc_idx;
    uint64_t m;                // accepted samples kept: min(accepted, capacity)
    const float* logq;         // the round's proposal log densities, NULL for prior draws
    uint64_t tail_first;       // first index of the defensive prior draws (UINT64_MAX: none)
    double* pool;              // the first pool_k weights go here (NULL: none)
    float* pool_theta;         // and the first pool_k samples' theta and distance
    double* pool_dist;
    uint64_t pool_k;
    float* train_theta;        // this round's training set (NULL: none): m rows in the
    float* train_w;            // order j -> (perm_a j + perm_b) mod m
    uint64_t perm_a, perm_b;
};

// per-region scratch of a round: positions over the round's n indices, block
// counts, the sorted samples, log weights, training weights, block sums
struct RegionScratch {
    uint32_t* pos;      // [R][n]
    uint32_t* count;    // [R][nb]
    float* theta;       // [R][cap][8]
    double* dist;       // [R][cap]
    uint64_t* idx;      // [R][cap]
    float* lw;          // [R][cap]
    float* w;           // [R][cap]
    double* bsum;       // [R][2 (cap / 256 + 1)]
    WeightScratch* ws;  // [R]
    uint64_t n, cap;
    uint32_t nb;
};

__device__ __forceinline__ bool region_block_in(uint64_t count)
{
    return (uint64_t)blockIdx.x * blockDim.x < count;
}

__global__ void scatter_slots_regions(const RegionRound* __restrict__ tab, uint64_t first, RegionScratch sc)
{
    const RegionRound& T = tab[blockIdx.y];
    if (!region_block_in(T.m)) return;
    scatter_slots_body(T.acc_idx, T.m, first, sc.pos + blockIdx.y * sc.n);
}

__global__ void __launch_bounds__(256) count_slots_regions(const RegionRound* __restrict__ tab, RegionScratch sc)
{
    if (tab[blockIdx.y].m == 0) return;
    count_slots_body(sc.pos + blockIdx.y * sc.n, sc.n, sc.count + (size_t)blockIdx.y * sc.nb);
}

__global__ void __launch_bounds__(256) scan_counts_regions(const RegionRound* __restrict__ tab, RegionScratch sc)
{
    if (tab[blockIdx.x].m == 0) return;
    scan_counts_body(sc.count + (size_t)blockIdx.x * sc.nb, sc.nb);
}

__global__ void __launch_bounds__(256) gather_sorted_regions(const RegionRound* __restrict__ tab, RegionScratch sc)
{
    const RegionRound& T = tab[blockIdx.y];
    if (T.m == 0) return;
    const size_t g = blockIdx.y;
    gather_sorted_body(sc.pos + g * sc.n, sc.n, sc.count + g * sc.nb, T.acc_theta, T.acc_dist, T.acc_idx,
                       sc.theta + g * sc.cap * 8, sc.dist + g * sc.cap, sc.idx + g * sc.cap);
}

__global__ void logw_regions(const RegionRound* __restrict__ tab, uint64_t first, float log_prior, RegionScratch sc)
{
    const RegionRound& T = tab[blockIdx.y];
    if (!region_block_in(T.m)) return;
    const size_t g = blockIdx.y;
    logw_body(T.logq, sc.idx + g * sc.cap, first, T.m, T.tail_first, log_prior, sc.lw + g * sc.cap, sc.ws + g);
}

__global__ void weight_regions(const RegionRound* __restrict__ tab, double power, RegionScratch sc)
{
    const RegionRound& T = tab[blockIdx.y];
    if (!region_block_in(T.m)) return;
    const size_t g = blockIdx.y;
    weight_body(sc.lw + g * sc.cap, T.m, sc.ws + g, sc.w + g * sc.cap, nullptr, T.pool, T.pool_k, power,
                sc.bsum + g * 2 * (sc.cap / 256 + 1));
}

__global__ void __launch_bounds__(256) weight_sums_regions(const RegionRound* __restrict__ tab, RegionScratch sc)
{
    const RegionRound& T = tab[blockIdx.x];
    if (T.m == 0) return;
    const size_t g = blockIdx.x;
    weight_sums_body(sc.bsum + g * 2 * (sc.cap / 256 + 1), (unsigned)((T.m + 255) / 256), sc.ws + g);
}

// the pooled samples (theta, distance) and this round's training set
__global__ void pool_and_train_regions(const RegionRound* __restrict__ tab, RegionScratch sc)
{
    const RegionRound& T = tab[blockIdx.y];
    const size_t g = blockIdx.y;
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float* th = sc.theta + g * sc.cap * 8;
    if (j < T.pool_k) {
        const float4* src = reinterpret_cast<const float4*>(th + 8 * j);
        float4* dst = reinterpret_cast<float4*>(T.pool_theta + 8 * j);
        dst[0] = src[0];
        dst[1] = src[1];
        T.pool_dist[j] = sc.dist[g * sc.cap + j];
    }
    if (T.train_theta && region_block_in(T.m))
        permute_body<float>(th, sc.w + g * sc.cap, T.m, T.m, T.perm_a, T.perm_b, T.train_theta, T.train_w);
}

// The second pass of a round, once the weight sums are on the host: each
// region's new pool weights scaled, then a training set drawn from its pool
struct RegionPool {
    double* w;                 // this round's pool weights, k of them, times f
    uint64_t k;
    double f;
    const float* theta;        // the pool: m samples and weights
    const double* pw;
    uint64_t m, n;             // n rows of training set (0: none) in the order j -> (a j + b) mod m
    uint64_t a, b;
    float* train_theta;
    float* train_w;
};

__global__ void scale_pools_regions(const RegionPool* __restrict__ tab)
{
    const RegionPool& T = tab[blockIdx.y];
    if (!region_block_in(T.k)) return;
    scale_body(T.w, T.k, T.f);
}

__global__ void train_from_pools_regions(const RegionPool* __restrict__ tab)
{
    const RegionPool& T = tab[blockIdx.y];
    if (!region_block_in(T.n)) return;
    permute_body<double>(T.theta, T.pw, T.m, T.n, T.a, T.b, T.train_theta, T.train_w);
}

struct Guard {
    std::vector<void*> dev;
    abc_plan plan = nullptr;
    abc_maf flow = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Guard()
    {
        for (void* p : dev) cudaFree(p);
        if (plan) abc_plan_destroy(plan);
        if (flow) abc_maf_destroy(flow);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace

using abcgb::plan_cuda_fail;
using abcgb::plan_fail;

#define SMC_TRY(expr, what)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return plan_cuda_fail(_e, what); \
    } while (0)
#define SMC_ST(expr)                        \
    do {                                    \
        abc_status _s = (expr);             \
        if (_s != ABC_OK) return _s;        \
    } while (0)

// The permutation j -> (a j + b) mod m of a training set: a near m times the
// golden ratio and coprime to m, b from the salt. m < 2^32.
static void perm_params(uint64_t m, uint64_t salt, uint64_t* a_out, uint64_t* b_out)
{
    uint64_t a = (uint64_t)(0.6180339887498949 * (double)m) | 1u;
    while (std::gcd(a, m) != 1) a += 2;
    *a_out = a % m ? a % m : 1;
    *b_out = (salt * 0x9E3779B97F4A7C15ull) % m;
}

// Shuffle m samples and their weights into a training set of the first
// n <= m of the permuted order (permute_kernel). m < 2^32.
template <typename W>
static abc_status shuffled_training_set(const float* theta, const W* w, uint64_t m, uint64_t n, uint64_t salt,
                                        float* theta_dst, float* w_dst, cudaStream_t s)
{
    uint64_t a = 0, b = 0;
    perm_params(m, salt, &a, &b);
    permute_kernel<W><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(theta, w, m, n, a, b, theta_dst, w_dst);
    SMC_TRY(cudaGetLastError(), "permute launch");
    return ABC_OK;
}

// Weights of a round's m accepted samples (logq: the round's proposal log
// densities, NULL for prior draws): float training weights v_j into w_train,
// optionally v_j in double into w_exact and the unnormalised weights of the
// first pool_k samples into pool; sum v, sum v^2 and the count of samples with
// index >= tail_first into *d_ws. Asynchronous on s.
// d_block_sums: 2 doubles per 256 samples.
static abc_status launch_round_weights(const float* logq, const uint64_t* idx, uint64_t first, uint64_t m,
                                       double log_prior, float* d_lw, float* w_train, double* w_exact, double* pool,
                                       uint64_t pool_k, WeightScratch* d_ws, double* d_block_sums, cudaStream_t s,
                                       double power, uint64_t tail_first)
{
    SMC_TRY(cudaMemsetAsync(d_ws, 0, sizeof(WeightScratch), s), "cudaMemsetAsync(weight scratch)");
    const unsigned blocks = (unsigned)((m + 255) / 256);
    logw_kernel<<<blocks, 256, 0, s>>>(logq, idx, first, m, tail_first, (float)log_prior, d_lw, d_ws);
    weight_kernel<<<blocks, 256, 0, s>>>(d_lw, m, d_ws, w_train, w_exact, pool, pool_k, power, d_block_sums);
    weight_sums_kernel<<<1, 256, 0, s>>>(d_block_sums, blocks, d_ws);
    SMC_TRY(cudaGetLastError(), "weight launch");
    return ABC_OK;
}

// launch_round_weights, then *sum_v, *sum_v2 and *n_tail read back.
// Synchronizes s.
static abc_status round_weights(const float* logq, const uint64_t* idx, uint64_t first, uint64_t m, double log_prior,
                                float* d_lw, float* w_train, double* w_exact, double* pool, uint64_t pool_k,
                                WeightScratch* d_ws, double* d_block_sums, cudaStream_t s, double* sum_v,
                                double* sum_v2, double power, uint64_t tail_first, uint64_t* n_tail)
{
    SMC_ST(launch_round_weights(logq, idx, first, m, log_prior, d_lw, w_train, w_exact, pool, pool_k, d_ws,
                                d_block_sums, s, power, tail_first));
    WeightScratch h;
    SMC_TRY(cudaMemcpyAsync(&h, d_ws, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(weight sums)");
    SMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *sum_v = h.sums[0];
    *sum_v2 = h.sums[1];
    *n_tail = h.n_tail;
    return ABC_OK;
}

// Device scratch of sort_accepted for runs of n sample indices and up to cap
// accepted samples, and of round_weights' block sums.
struct SortScratch {
    uint32_t* pos = nullptr;     // [n]
    uint32_t* count = nullptr;   // [n / 1024 + 1]
    float* theta = nullptr;      // [cap][8], the sorted samples
    double* dist = nullptr;      // [cap]
    uint64_t* idx = nullptr;     // [cap]
    double* block_sums = nullptr;   // [2 (cap / 256 + 1)]
};

static abc_status alloc_sort_scratch(SortScratch& sc, uint64_t n, uint64_t cap, std::vector<void*>& owned)
{
    const uint64_t nb = (n + kSortBlock - 1) / kSortBlock + 1;
    SMC_TRY(cudaMalloc(&sc.pos, sizeof(uint32_t) * n), "cudaMalloc(sort positions)");
    owned.push_back(sc.pos);
    SMC_TRY(cudaMalloc(&sc.count, sizeof(uint32_t) * nb), "cudaMalloc(sort counts)");
    owned.push_back(sc.count);
    SMC_TRY(cudaMalloc(&sc.theta, sizeof(float) * 8 * cap), "cudaMalloc(sorted theta)");
    owned.push_back(sc.theta);
    SMC_TRY(cudaMalloc(&sc.dist, sizeof(double) * cap), "cudaMalloc(sorted dist)");
    owned.push_back(sc.dist);
    SMC_TRY(cudaMalloc(&sc.idx, sizeof(uint64_t) * cap), "cudaMalloc(sorted idx)");
    owned.push_back(sc.idx);
    SMC_TRY(cudaMalloc(&sc.block_sums, sizeof(double) * 2 * (cap / 256 + 1)), "cudaMalloc(weight block sums)");
    owned.push_back(sc.block_sums);
    return ABC_OK;
}

// The m accepted samples of a run over indices [first, first + n) into
// sc.theta, sc.dist, sc.idx in ascending index (the kernels above). Async.
static abc_status sort_accepted(const float* theta, const double* dist, const uint64_t* idx, uint64_t m, uint64_t first,
                                uint64_t n, SortScratch& sc, cudaStream_t s)
{
    if (m == 0) return ABC_OK;
    const uint32_t nb = (uint32_t)((n + kSortBlock - 1) / kSortBlock);
    SMC_TRY(cudaMemsetAsync(sc.pos, 0xFF, sizeof(uint32_t) * n, s), "cudaMemsetAsync(sort positions)");
    scatter_slots_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(idx, m, first, sc.pos);
    count_slots_kernel<<<nb, 256, 0, s>>>(sc.pos, n, sc.count);
    scan_counts_kernel<<<1, 256, 0, s>>>(sc.count, nb);
    gather_sorted_kernel<<<nb, 256, 0, s>>>(sc.pos, n, sc.count, theta, dist, idx, sc.theta, sc.dist, sc.idx);
    SMC_TRY(cudaGetLastError(), "sort launch");
    return ABC_OK;
}

// Whether the next round should draw from the flow. By efficiency: a flow
// round keeps the flow when it gave at least as many effective samples per
// simulation, ESS / N with ESS = (sum w)^2 / sum w^2, as rejection from the
// prior accepts per simulation at the same eps, that rate measured on the
// round's own defensive prior draws; a prior round, or a flow round without
// defensive draws, keeps or switches to the flow when its ESS fraction
// reaches ess_min. By ESS: every round by its ESS fraction. Fewer than 64
// accepted samples always means the prior.
static bool next_uses_flow(const abc_smc_round& R, double sw, double sw2, const abc_smc_config& cfg)
{
    if (R.n_accepted < 64 || !(sw2 > 0.0)) return false;
    if (cfg.fallback_rule == ABC_FALLBACK_ESS || R.proposal == 0 || R.n_defensive == 0)
        return R.ess_fraction >= cfg.ess_min;
    return sw * sw / sw2 / (double)R.n_sims >= (double)R.n_defensive_accepted / (double)R.n_defensive;
}

extern "C" abc_status abc_smc_run(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                                  const abc_smc_config* cfg, abc_smc_round* rounds_out, float* theta_out,
                                  double* weight_out, double* dist_out, uint64_t* n_out, void* cuda_stream)
{
    abc_status st;
    if (!abcgb::plan_check_prior(prior, &st)) return st;
    if (!cfg || !rounds_out || !n_out) return plan_fail(ABC_ERR_INVALID_ARG, "cfg, rounds_out and n_out are required");
    if (cfg->rounds < 1 || cfg->sims_per_round == 0 || !(cfg->eps0 >= 0.0) || !(cfg->eps_factor > 0.0) ||
        cfg->eps_factor > 1.0 || !(cfg->ess_min >= 0.0) || cfg->capacity == 0 || !(cfg->defensive >= 0.0) ||
        cfg->defensive >= 1.0 || !(cfg->val_fraction >= 0.0) || cfg->val_fraction > 0.5 ||
        !(cfg->train_weight_power > 0.0) || cfg->train_weight_power > 1.0 || !(cfg->proposal_scale >= 0.5) ||
        cfg->proposal_scale > 4.0 || (cfg->fallback_rule != ABC_FALLBACK_EFFICIENCY && cfg->fallback_rule != ABC_FALLBACK_ESS))
        return plan_fail(ABC_ERR_INVALID_ARG, "bad sequential ABC configuration");
    // every accepted sample of a round is kept: the accept buffer is filled in
    // claim (index) order and a flow round's defensive prior draws are its
    // last indices, so a truncated round would drop them selectively
    if (cfg->capacity < cfg->sims_per_round)
        return plan_fail(ABC_ERR_INVALID_ARG, "capacity must be >= sims_per_round");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s) return plan_fail(ABC_ERR_INVALID_ARG, "sequential ABC needs a non-default stream");
    const uint64_t N = cfg->sims_per_round, cap = cfg->capacity;
    double log_prior = 0.0;
    for (int j = 0; j < 8; ++j) log_prior -= std::log((double)prior->hi[j] - (double)prior->lo[j]);

    Guard gd;
    SMC_ST(abc_maf_create(cfg->flow_blocks, cfg->flow_hidden, prior, &gd.flow));
    SMC_ST(abc_maf_set_proposal_scale(gd.flow, (float)cfg->proposal_scale));
    SMC_ST(abc_maf_init_random(gd.flow, cfg->seed ^ 0x5EED5EEDull, 0.3f));
    float *d_prop = nullptr, *d_logq = nullptr, *d_acc_logq = nullptr, *d_w = nullptr;
    SMC_TRY(cudaMalloc(&d_prop, sizeof(float) * 8 * N), "cudaMalloc(proposals)");
    gd.dev.push_back(d_prop);
    SMC_TRY(cudaMalloc(&d_logq, sizeof(float) * N), "cudaMalloc(logq)");
    gd.dev.push_back(d_logq);
    SMC_TRY(cudaMalloc(&d_acc_logq, sizeof(float) * cap), "cudaMalloc(log weights)");
    gd.dev.push_back(d_acc_logq);
    SMC_TRY(cudaMalloc(&d_w, sizeof(float) * cap), "cudaMalloc(weights)");
    gd.dev.push_back(d_w);
    WeightScratch* d_ws = nullptr;
    SMC_TRY(cudaMalloc(&d_ws, sizeof(WeightScratch)), "cudaMalloc(weight scratch)");
    gd.dev.push_back(d_ws);
    float* d_wround = nullptr;
    SMC_TRY(cudaMalloc(&d_wround, sizeof(float) * cap), "cudaMalloc(round weights)");
    gd.dev.push_back(d_wround);
    float* d_train = nullptr;
    SMC_TRY(cudaMalloc(&d_train, sizeof(float) * 8 * cap), "cudaMalloc(training set)");
    gd.dev.push_back(d_train);
    SortScratch ss;
    SMC_ST(alloc_sort_scratch(ss, N, cap, gd.dev));
    for (cudaEvent_t& e : gd.ev) SMC_TRY(cudaEventCreate(&e), "cudaEventCreate");

    double eps = cfg->eps0;
    bool use_flow = false;
    uint64_t last_n = 0;
    // one plan for every round, made before the first; each round sets its
    // eps, proposals and first index before its timed stages
    {
        abc_region reg{};
        reg.observed = observed;
        reg.T = T;
        reg.N_pop = N_pop;
        reg.eps = eps;
        reg.n_samples = N;
        reg.first_index = 0;
        reg.stream = 0;
        reg.capacity = cap;
        reg.theta_in = nullptr;
        SMC_ST(abc_plan_create(prior, &reg, 1, cfg->seed, cfg->mode, &gd.plan));
    }
    for (int32_t r = 0; r < cfg->rounds; ++r) {
        abc_smc_round& R = rounds_out[r];
        R = abc_smc_round{};
        R.eps = eps;
        R.proposal = use_flow ? 1 : 0;
        R.n_sims = N;
        const uint64_t first = (uint64_t)r * N;
        SMC_ST(abc_plan_set_eps(gd.plan, 0, eps));
        SMC_ST(abc_plan_set_region(gd.plan, 0, use_flow ? d_prop : nullptr, first));
        SMC_TRY(cudaEventRecord(gd.ev[0], s), "cudaEventRecord");
        if (use_flow) {
            // (1 - defensive) N flow draws, the rest prior draws, all weighted by the mixture density
            const uint64_t n_prior = (uint64_t)std::floor(cfg->defensive * (double)N);
            const uint64_t n_flow = N - n_prior;
            R.n_defensive = n_prior;
            // flow draws carry the sampler's log q (exact for the drawn point); the
            // prior draws get the flow's density evaluated at them
            if (n_flow) SMC_ST(abc_maf_sample(gd.flow, n_flow, nullptr, cfg->seed, 1, first, d_prop, d_logq, s));
            if (n_prior) {
                const abcgb::ModelParams pp = abcgb::plan_make_params(prior, 1, 1, cfg->seed, 0, nullptr);
                prior_theta_kernel<<<(unsigned)((n_prior + 255) / 256), 256, 0, s>>>(pp, first + n_flow, n_prior,
                                                                                   d_prop + 8 * n_flow);
                SMC_TRY(cudaGetLastError(), "prior draw launch");
                SMC_ST(abc_maf_log_q(gd.flow, n_prior, d_prop + 8 * n_flow, d_logq + n_flow, s));
            }
            if (cfg->defensive > 0.0) {
                mixture_logq_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
                    d_logq, N, (float)std::log1p(-cfg->defensive), (float)(std::log(cfg->defensive) + log_prior));
                SMC_TRY(cudaGetLastError(), "mixture launch");
            }
        }
        SMC_TRY(cudaEventRecord(gd.ev[1], s), "cudaEventRecord");
        SMC_ST(abc_plan_reset(gd.plan, s));
        SMC_ST(abc_plan_run(gd.plan, s));
        SMC_TRY(cudaEventRecord(gd.ev[2], s), "cudaEventRecord");
        uint64_t n_acc = 0, days = 0;
        float* acc_theta = nullptr;
        double* acc_dist = nullptr;
        uint64_t* acc_idx = nullptr;
        SMC_ST(abc_plan_results(gd.plan, 0, &n_acc, &days, &acc_theta, &acc_dist, &acc_idx, s));
        R.n_accepted = n_acc;
        R.simulated_days = days;
        const uint64_t m = std::min(n_acc, cap);
        // the accepted samples in index order, the same in every run
        SMC_ST(sort_accepted(acc_theta, acc_dist, acc_idx, m, first, N, ss, s));
        acc_theta = ss.theta;
        acc_dist = ss.dist;
        acc_idx = ss.idx;
        const bool last = r + 1 == cfg->rounds;
        // importance weights prior / q_mix of the kept accepted samples
        double sw = 0.0, sw2 = 0.0;
        if (m > 0) {
            // a flow round's defensive prior draws are its last n_defensive indices
            const uint64_t tail_first = use_flow ? first + N - R.n_defensive : UINT64_MAX;
            uint64_t n_tail = 0;
            SMC_ST(round_weights(use_flow ? d_logq : nullptr, acc_idx, first, m, log_prior, d_acc_logq, d_wround,
                                 last ? weight_out : nullptr, nullptr, 0, d_ws, ss.block_sums, s, &sw, &sw2,
                                 cfg->train_weight_power, tail_first, &n_tail));
            R.ess_fraction = sw2 > 0.0 ? sw * sw / sw2 / (double)m : 0.0;
            R.n_defensive_accepted = n_tail;
        }
        // the next round's proposal: train on this round's weighted accepts
        if (last) {
            last_n = m;
            if (m > 0) {
                if (theta_out)
                    SMC_TRY(cudaMemcpyAsync(theta_out, acc_theta, sizeof(float) * 8 * m, cudaMemcpyDefault, s),
                            "cudaMemcpyAsync(theta)");
                if (dist_out)
                    SMC_TRY(cudaMemcpyAsync(dist_out, acc_dist, sizeof(double) * m, cudaMemcpyDefault, s),
                            "cudaMemcpyAsync(dist)");
                if (weight_out && sw > 0.0) {
                    scale_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(weight_out, m, 1.0 / sw);
                    SMC_TRY(cudaGetLastError(), "scale launch");
                }
            }
            SMC_TRY(cudaEventRecord(gd.ev[3], s), "cudaEventRecord");
        } else {
            const bool trainable = next_uses_flow(R, sw, sw2, *cfg);
            if (trainable) {
                SMC_ST(shuffled_training_set(acc_theta, d_wround, m, m, cfg->seed + (uint64_t)r, d_train, d_w, s));
                if (cfg->fresh_init)
                    SMC_ST(abc_maf_init_random(gd.flow, (cfg->seed ^ 0x5EED5EEDull) + 7 * (uint64_t)(r + 1), 0.3f));
                float loss = 0.f;
                const float* tt = d_train;
                const float* tw = d_w;
                const uint64_t tn = m;
                SMC_ST(abc_maf_train_flows(gd.flow, &tt, &tw, &tn, cfg->train_steps, cfg->train_batch, cfg->train_lr,
                                           cfg->seed + 7919 * (uint64_t)r, (float)cfg->val_fraction, &loss, s));
                R.train_loss = loss;
            }
            SMC_TRY(cudaEventRecord(gd.ev[3], s), "cudaEventRecord");
            use_flow = trainable;
        }
        SMC_TRY(cudaEventSynchronize(gd.ev[3]), "cudaEventSynchronize");
        cudaEventElapsedTime(&R.ms_propose, gd.ev[0], gd.ev[1]);
        cudaEventElapsedTime(&R.ms_simulate, gd.ev[1], gd.ev[2]);
        cudaEventElapsedTime(&R.ms_train, gd.ev[2], gd.ev[3]);
        eps *= cfg->eps_factor;
    }
    SMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *n_out = last_n;
    return abcgb::plan_ok();
}

namespace {

struct RegionsGuard {
    std::vector<void*> dev;
    abc_plan plan = nullptr;
    abc_maf flows = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~RegionsGuard()
    {
        for (void* p : dev) cudaFree(p);
        if (plan) abc_plan_destroy(plan);
        if (flows) abc_maf_destroy(flows);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace

extern "C" abc_status abc_smc_run_regions(const abc_prior_box* prior, abc_smc_region* regions, int32_t n_regions,
                                          const abc_smc_stream_config* scfg, abc_smc_round* rounds_out,
                                          void* cuda_stream)
{
    abc_status st;
    if (!abcgb::plan_check_prior(prior, &st)) return st;
    if (!scfg || !rounds_out || !regions) return plan_fail(ABC_ERR_INVALID_ARG, "regions, cfg and rounds_out are required");
    const abc_smc_config* cfg = &scfg->base;
    const int32_t R = n_regions;
    if (R < 1 || R > ABC_MAX_REGIONS) return plan_fail(ABC_ERR_INVALID_ARG, "n_regions must be in [1, ABC_MAX_REGIONS]");
    if (cfg->rounds < 1 || cfg->sims_per_round == 0 || !(cfg->eps_factor > 0.0) || cfg->eps_factor > 1.0 ||
        !(cfg->ess_min >= 0.0) || cfg->capacity == 0 || !(cfg->defensive >= 0.0) || cfg->defensive >= 1.0 ||
        !(cfg->val_fraction >= 0.0) || cfg->val_fraction > 0.5 || cfg->capacity < cfg->sims_per_round ||
        !(cfg->train_weight_power > 0.0) || cfg->train_weight_power > 1.0 || !(cfg->proposal_scale >= 0.5) ||
        cfg->proposal_scale > 4.0 ||
        (cfg->fallback_rule != ABC_FALLBACK_EFFICIENCY && cfg->fallback_rule != ABC_FALLBACK_ESS) || scfg->shrink_rounds < 1 || scfg->shrink_rounds > cfg->rounds || scfg->train_steps_warm < 0 ||
        cfg->train_steps < 0)
        return plan_fail(ABC_ERR_INVALID_ARG, "bad multi-region sequential ABC configuration");
    for (int32_t g = 0; g < R; ++g) {
        const abc_smc_region& G = regions[g];
        if (!G.observed || !(G.eps >= 0.0)) return plan_fail(ABC_ERR_INVALID_ARG, "a region lacks observed data or eps");
        if (G.capacity > 0 && (!G.theta_out || !G.weight_out || !G.dist_out))
            return plan_fail(ABC_ERR_INVALID_ARG, "a region with capacity > 0 lacks output buffers");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s) return plan_fail(ABC_ERR_INVALID_ARG, "sequential ABC needs a non-default stream");
    const uint64_t N = cfg->sims_per_round, cap = cfg->capacity;
    const int32_t S = scfg->shrink_rounds;
    double log_prior = 0.0;
    for (int j = 0; j < 8; ++j) log_prior -= std::log((double)prior->hi[j] - (double)prior->lo[j]);

    RegionsGuard gd;
    SMC_ST(abc_maf_create_multi(R, cfg->flow_blocks, cfg->flow_hidden, prior, &gd.flows));
    SMC_ST(abc_maf_set_proposal_scale(gd.flows, (float)cfg->proposal_scale));
    SMC_ST(abc_maf_init_random(gd.flows, cfg->seed ^ 0x5EED5EEDull, 0.3f));
    float *d_prop = nullptr, *d_logq = nullptr, *d_w = nullptr, *d_train = nullptr;
    SMC_TRY(cudaMalloc(&d_prop, sizeof(float) * 8 * N * R), "cudaMalloc(proposals)");
    gd.dev.push_back(d_prop);
    SMC_TRY(cudaMalloc(&d_logq, sizeof(float) * N * R), "cudaMalloc(logq)");
    gd.dev.push_back(d_logq);
    SMC_TRY(cudaMalloc(&d_w, sizeof(float) * cap * R), "cudaMalloc(weights)");
    gd.dev.push_back(d_w);
    SMC_TRY(cudaMalloc(&d_train, sizeof(float) * 8 * cap * R), "cudaMalloc(training sets)");
    gd.dev.push_back(d_train);
    // per-region scratch of a round's results (RegionScratch) and the tables
    // of the two passes
    RegionScratch rs{};
    rs.n = N;
    rs.cap = cap;
    rs.nb = (uint32_t)((N + kSortBlock - 1) / kSortBlock);
    {
        const size_t Rz = (size_t)R;
        void* q = nullptr;
        auto grab = [&](size_t bytes, const char* what) -> abc_status {
            SMC_TRY(cudaMalloc(&q, bytes), what);
            gd.dev.push_back(q);
            return ABC_OK;
        };
        SMC_ST(grab(sizeof(uint32_t) * N * Rz, "cudaMalloc(sort positions)"));
        rs.pos = (uint32_t*)q;
        SMC_ST(grab(sizeof(uint32_t) * rs.nb * Rz, "cudaMalloc(sort counts)"));
        rs.count = (uint32_t*)q;
        SMC_ST(grab(sizeof(float) * 8 * cap * Rz, "cudaMalloc(sorted theta)"));
        rs.theta = (float*)q;
        SMC_ST(grab(sizeof(double) * cap * Rz, "cudaMalloc(sorted dist)"));
        rs.dist = (double*)q;
        SMC_ST(grab(sizeof(uint64_t) * cap * Rz, "cudaMalloc(sorted idx)"));
        rs.idx = (uint64_t*)q;
        SMC_ST(grab(sizeof(float) * cap * Rz, "cudaMalloc(log weights)"));
        rs.lw = (float*)q;
        SMC_ST(grab(sizeof(float) * cap * Rz, "cudaMalloc(round weights)"));
        rs.w = (float*)q;
        SMC_ST(grab(sizeof(double) * 2 * (cap / 256 + 1) * Rz, "cudaMalloc(weight block sums)"));
        rs.bsum = (double*)q;
        SMC_ST(grab(sizeof(WeightScratch) * Rz, "cudaMalloc(weight scratch)"));
        rs.ws = (WeightScratch*)q;
    }
    RegionRound* d_rr = nullptr;
    RegionPool* d_rp = nullptr;
    SMC_TRY(cudaMalloc(&d_rr, sizeof(RegionRound) * R), "cudaMalloc(round table)");
    gd.dev.push_back(d_rr);
    SMC_TRY(cudaMalloc(&d_rp, sizeof(RegionPool) * R), "cudaMalloc(pool table)");
    gd.dev.push_back(d_rp);
    for (cudaEvent_t& e : gd.ev) SMC_TRY(cudaEventCreate(&e), "cudaEventCreate");

    // one plan for every round: the regions' eps, proposals and first indices
    // are set before each run
    std::vector<abc_region> regs((size_t)R);
    for (int32_t g = 0; g < R; ++g) {
        abc_region& q = regs[g];
        q = abc_region{};
        q.observed = regions[g].observed;
        q.T = regions[g].T;
        q.N_pop = regions[g].N_pop;
        q.eps = regions[g].eps;
        q.n_samples = N;
        q.first_index = 0;
        q.stream = (uint32_t)g;
        q.capacity = cap;
        q.theta_in = nullptr;
        regions[g].n_pooled = 0;
        regions[g].n_out = 0;
    }
    SMC_ST(abc_plan_create(prior, regs.data(), R, cfg->seed, cfg->mode, &gd.plan));

    std::vector<char> use_flow((size_t)R, 0), trainable((size_t)R, 0), next_flow((size_t)R, 0);
    bool trained_once = false;
    std::vector<float> losses((size_t)R, 0.f);
    std::vector<const float*> tr_theta((size_t)R), tr_w((size_t)R);
    std::vector<uint64_t> tr_n((size_t)R);
    for (int32_t r = 0; r < cfg->rounds; ++r) {
        const uint64_t first = (uint64_t)r * N;
        abc_smc_round* Rr = rounds_out + (size_t)r * R;
        SMC_TRY(cudaEventRecord(gd.ev[0], s), "cudaEventRecord");
        for (int32_t g = 0; g < R; ++g) {
            const double eps = r < S ? regions[g].eps / std::pow(cfg->eps_factor, (double)(S - 1 - r)) : regions[g].eps;
            Rr[g] = abc_smc_round{};
            Rr[g].eps = eps;
            Rr[g].proposal = use_flow[g] ? 1 : 0;
            Rr[g].n_sims = N;
            if (use_flow[g]) {
                const uint64_t n_prior = (uint64_t)std::floor(cfg->defensive * (double)N);
                const uint64_t n_flow = N - n_prior;
                Rr[g].n_defensive = n_prior;
                float* prop = d_prop + (size_t)g * 8 * N;
                float* lq = d_logq + (size_t)g * N;
                if (n_flow)
                    SMC_ST(abc_maf_sample_at(gd.flows, g, n_flow, nullptr, cfg->seed, (uint32_t)(R + g), first, prop, lq,
                                             s));
                if (n_prior) {
                    const abcgb::ModelParams pp = abcgb::plan_make_params(prior, 1, 1, cfg->seed, (uint32_t)g, nullptr);
                    prior_theta_kernel<<<(unsigned)((n_prior + 255) / 256), 256, 0, s>>>(pp, first + n_flow, n_prior,
                                                                                       prop + 8 * n_flow);
                    SMC_TRY(cudaGetLastError(), "prior draw launch");
                    SMC_ST(abc_maf_log_q_at(gd.flows, g, n_prior, prop + 8 * n_flow, lq + n_flow, s));
                }
                if (cfg->defensive > 0.0) {
                    mixture_logq_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
                        lq, N, (float)std::log1p(-cfg->defensive), (float)(std::log(cfg->defensive) + log_prior));
                    SMC_TRY(cudaGetLastError(), "mixture launch");
                }
            }
            SMC_ST(abc_plan_set_eps(gd.plan, g, eps));
            SMC_ST(abc_plan_set_region(gd.plan, g, use_flow[g] ? d_prop + (size_t)g * 8 * N : nullptr, first));
        }
        SMC_TRY(cudaEventRecord(gd.ev[1], s), "cudaEventRecord");
        SMC_ST(abc_plan_reset(gd.plan, s));
        SMC_ST(abc_plan_run(gd.plan, s));
        SMC_TRY(cudaEventRecord(gd.ev[2], s), "cudaEventRecord");
        // The regions' results in two passes with one synchronisation between
        // them, every step one launch over all regions (grid row = region):
        // first the accepted samples in index order, their weights (the sums
        // kept on the device), the copies into the pool and this round's
        // training set; then, with all regions' weight sums read back at
        // once, what depends on them (the ESS, the pool's scale, the next
        // proposal, a training set from the pool).
        bool any_train = false;
        std::vector<uint64_t> n_acc_v((size_t)R), days_v((size_t)R), k_v((size_t)R, 0);
        std::vector<float*> th_v((size_t)R);
        std::vector<double*> di_v((size_t)R);
        std::vector<uint64_t*> ix_v((size_t)R);
        SMC_ST(abcgb::plan_results_all(gd.plan, n_acc_v.data(), days_v.data(), th_v.data(), di_v.data(), ix_v.data(),
                                       s));
        const bool pool = r >= S - 1;
        const bool round_sets = !pool && r + 1 < cfg->rounds;   // training sets from this round alone
        std::vector<RegionRound> rr((size_t)R);
        uint64_t max_m = 0, max_k = 0;
        for (int32_t g = 0; g < R; ++g) {
            Rr[g].n_accepted = n_acc_v[g];
            Rr[g].simulated_days = days_v[g];
            trainable[g] = 0;
            next_flow[g] = 0;
            tr_n[g] = 0;
            RegionRound& T = rr[g];
            T = RegionRound{};
            T.m = std::min(n_acc_v[g], cap);
            if (T.m == 0) continue;
            abc_smc_region& G = regions[g];
            T.acc_theta = th_v[g];
            T.acc_dist = di_v[g];
            T.acc_idx = ix_v[g];
            // weights prior / q_mix (1 for prior draws); a flow round's
            // defensive prior draws are its last n_defensive indices
            T.logq = use_flow[g] ? d_logq + (size_t)g * N : nullptr;
            T.tail_first = use_flow[g] ? first + N - Rr[g].n_defensive : UINT64_MAX;
            T.pool_k = k_v[g] = pool ? std::min(T.m, G.capacity - G.n_out) : 0;
            if (T.pool_k) {
                T.pool = G.weight_out + G.n_out;
                T.pool_theta = G.theta_out + 8 * G.n_out;
                T.pool_dist = G.dist_out + G.n_out;
            }
            // before the final eps the flow trains on this round's weighted
            // accepts, if the weights show it worth it (decided below)
            if (round_sets) {
                T.train_theta = d_train + (size_t)g * 8 * cap;
                T.train_w = d_w + (size_t)g * cap;
                perm_params(T.m, cfg->seed + 131 * (uint64_t)r + (uint64_t)g, &T.perm_a, &T.perm_b);
            }
            max_m = std::max(max_m, T.m);
            max_k = std::max(max_k, T.pool_k);
        }
        if (max_m > 0) {
            const unsigned Ru = (unsigned)R, mb = (unsigned)((max_m + 255) / 256);
            SMC_TRY(cudaMemcpyAsync(d_rr, rr.data(), sizeof(RegionRound) * R, cudaMemcpyHostToDevice, s),
                    "cudaMemcpyAsync(round table)");
            // the accepted samples in index order, the same in every run
            SMC_TRY(cudaMemsetAsync(rs.pos, 0xFF, sizeof(uint32_t) * N * R, s), "cudaMemsetAsync(sort positions)");
            scatter_slots_regions<<<dim3(mb, Ru), 256, 0, s>>>(d_rr, first, rs);
            count_slots_regions<<<dim3(rs.nb, Ru), 256, 0, s>>>(d_rr, rs);
            scan_counts_regions<<<Ru, 256, 0, s>>>(d_rr, rs);
            gather_sorted_regions<<<dim3(rs.nb, Ru), 256, 0, s>>>(d_rr, rs);
            SMC_TRY(cudaGetLastError(), "sort launch");
            SMC_TRY(cudaMemsetAsync(rs.ws, 0, sizeof(WeightScratch) * R, s), "cudaMemsetAsync(weight scratch)");
            logw_regions<<<dim3(mb, Ru), 256, 0, s>>>(d_rr, first, (float)log_prior, rs);
            weight_regions<<<dim3(mb, Ru), 256, 0, s>>>(d_rr, cfg->train_weight_power, rs);
            weight_sums_regions<<<Ru, 256, 0, s>>>(d_rr, rs);
            if (max_k > 0 || round_sets)
                pool_and_train_regions<<<dim3((unsigned)((std::max(max_k, round_sets ? max_m : 0) + 255) / 256), Ru),
                                         256, 0, s>>>(d_rr, rs);
            SMC_TRY(cudaGetLastError(), "weight launch");
        }
        std::vector<WeightScratch> hws((size_t)R);
        if (max_m > 0)
            SMC_TRY(cudaMemcpyAsync(hws.data(), rs.ws, sizeof(WeightScratch) * R, cudaMemcpyDeviceToHost, s),
                    "cudaMemcpyAsync(weight sums)");
        SMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        std::vector<RegionPool> rp((size_t)R);
        uint64_t max_scale = 0, max_set = 0;
        for (int32_t g = 0; g < R; ++g) {
            rp[g] = RegionPool{};
            const uint64_t n_acc = n_acc_v[g], m = std::min(n_acc, cap);
            if (m == 0) continue;
            abc_smc_region& G = regions[g];
            const uint64_t k = k_v[g];
            const double sw = hws[g].sums[0], sw2 = hws[g].sums[1];
            Rr[g].ess_fraction = sw2 > 0.0 ? sw * sw / sw2 / (double)m : 0.0;
            Rr[g].n_defensive_accepted = hws[g].n_tail;
            // samples accepted at the region's final eps join the pool; the
            // rounds' self-normalised estimates are combined with weights
            // proportional to their ESS, i.e. sample weight v_j sum v / sum v^2
            if (pool) {
                G.n_pooled += n_acc;
                if (k > 0) {
                    rp[g].w = G.weight_out + G.n_out;
                    rp[g].k = k;
                    rp[g].f = sw / sw2;
                    max_scale = std::max(max_scale, k);
                    G.n_out += k;
                }
            }
            // the next round uses the flow unless the prior does better
            // (next_uses_flow); the flow trains on this round's weighted
            // accepts, or, once at the final eps, on the whole pool (same
            // target, more points)
            const bool good = next_uses_flow(Rr[g], sw, sw2, *cfg);
            if (r + 1 < cfg->rounds) {
                float* tt = d_train + (size_t)g * 8 * cap;
                float* tw = d_w + (size_t)g * cap;
                uint64_t tn = 0;
                if (pool && G.n_out >= 64) {
                    tn = std::min(G.n_out, cap);
                    RegionPool& P = rp[g];
                    P.theta = G.theta_out;
                    P.pw = G.weight_out;
                    P.m = G.n_out;
                    P.n = tn;
                    perm_params(G.n_out, cfg->seed + 131 * (uint64_t)r + (uint64_t)g, &P.a, &P.b);
                    P.train_theta = tt;
                    P.train_w = tw;
                    max_set = std::max(max_set, tn);
                } else if (!pool && good) {
                    tn = m;   // built above
                }
                if (tn > 0) {
                    trainable[g] = 1;
                    tr_theta[g] = tt;
                    tr_w[g] = tw;
                    tr_n[g] = tn;
                    any_train = true;
                }
            }
            next_flow[g] = good && (trainable[g] || use_flow[g]);
        }
        if (max_scale > 0 || max_set > 0) {
            SMC_TRY(cudaMemcpyAsync(d_rp, rp.data(), sizeof(RegionPool) * R, cudaMemcpyHostToDevice, s),
                    "cudaMemcpyAsync(pool table)");
            // the scaled weights first: a training set from the pool reads them
            if (max_scale > 0)
                scale_pools_regions<<<dim3((unsigned)((max_scale + 255) / 256), (unsigned)R), 256, 0, s>>>(d_rp);
            if (max_set > 0)
                train_from_pools_regions<<<dim3((unsigned)((max_set + 255) / 256), (unsigned)R), 256, 0, s>>>(d_rp);
            SMC_TRY(cudaGetLastError(), "pool launch");
        }
        if (any_train) {
            const int32_t steps = trained_once ? scfg->train_steps_warm : cfg->train_steps;
            SMC_ST(abc_maf_train_flows(gd.flows, tr_theta.data(), tr_w.data(), tr_n.data(), steps, cfg->train_batch,
                                       cfg->train_lr, cfg->seed + 7919 * (uint64_t)r, (float)cfg->val_fraction,
                                       losses.data(), s));
            trained_once = true;
            for (int32_t g = 0; g < R; ++g)
                if (trainable[g]) Rr[g].train_loss = losses[g];
        }
        SMC_TRY(cudaEventRecord(gd.ev[3], s), "cudaEventRecord");
        SMC_TRY(cudaEventSynchronize(gd.ev[3]), "cudaEventSynchronize");
        float ms[3] = {0.f, 0.f, 0.f};
        cudaEventElapsedTime(&ms[0], gd.ev[0], gd.ev[1]);
        cudaEventElapsedTime(&ms[1], gd.ev[1], gd.ev[2]);
        cudaEventElapsedTime(&ms[2], gd.ev[2], gd.ev[3]);
        for (int32_t g = 0; g < R; ++g) {
            Rr[g].ms_propose = ms[0];
            Rr[g].ms_simulate = ms[1];
            Rr[g].ms_train = ms[2];
            use_flow[g] = next_flow[g];
        }
    }
    SMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return abcgb::plan_ok();
}
