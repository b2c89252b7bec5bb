// abc_kernels.cu -- sm_103a kernels of ABC rejection sampling (paper Sec. 2.2,
// Sec. 3.1): one simulation per thread, the compartments in registers, the
// observed series in shared memory, the accepted samples compacted with a
// warp ballot and one atomic per warp.
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <cuda_runtime.h>

#include "abc_kernels.h"
#include "abc_model.cuh"

namespace abcgb {

// Stage the observed (A, R, D, 0) series of days 0..T into shared memory.
__device__ __forceinline__ void stage_observed(int4* obs_s, const int4* __restrict__ obs, int32_t T)
{
    for (int32_t d = threadIdx.x; d <= T; d += blockDim.x) obs_s[d] = obs[d];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// K1: fused rejection with early rejection and lane refill.
//
// The partial sums of the distance^2 only grow, so a sample whose running sum
// exceeds acc_max after some day pair can never be accepted: its lane drops it
// and takes the next sample (the accept set and the accepted distances are
// exactly those of running every sample for all T days). Each warp keeps a
// 64-entry ring of prior draws in shared memory, refilled 32 at a time by the
// whole warp (sample indices claimed with one atomicAdd per 32), so the theta
// draw of a new sample costs one shared-memory read for the lane that needs
// it. The loop advances every active lane by one day pair; all ring
// bookkeeping is warp-uniform. A ring entry holds the sample's parameters as
// the day loop uses them and its initial I0, worked out when the ring is
// refilled (32 samples, one per lane), so handing a sample to an idle lane
// is a few shared-memory reads. Accepted samples are compacted with a ballot
// and one atomicAdd per warp; their theta is re-drawn from the index.
// ---------------------------------------------------------------------------
constexpr int kRing = 64;
constexpr int kWarpsPerBlock = kBlockThreads / 32;
// A warp hands new samples to its idle lanes once at least kRefillMinIdle of
// them are idle (all 32 always qualify): the hand-out (ring read, derived
// parameters, initial state) runs on the whole warp, while a lane left idle
// for a day pair costs a 32nd of one. Measured on P = 6e7, T = 100, 2^24
// samples: 5.67 ms per launch at 1, 5.58 at 2 and at 4, 5.84 at 8. Which lane
// runs a sample, and when, does not change the sample's result.
constexpr uint32_t kRefillMinIdle = 2;

struct WarpRing {
    float4 lo[kRing];     // Theta a0, a, n, beta
    float4 hi[kRing];     // Theta gamma, delta, beta_eta; I0 (int32 bits)
    uint64_t idx[kRing];  // sample index
};

// Ring entry of sample ii: its Theta (kappa folded into I0) and I0.
template <int MODE>
__device__ __forceinline__ void ring_put(WarpRing& ring, uint32_t slot, const ModelParams& p, uint64_t ii,
                                         const float th[8], int32_t A0, int32_t room)
{
    const Theta t = make_theta<MODE>(th, p.inv_p);
    const int32_t I0 = initial_infected(t, A0, room);
    ring.lo[slot] = make_float4(t.a0, t.a, t.n, t.beta);
    ring.hi[slot] = make_float4(t.gamma, t.delta, t.beta_eta, __int_as_float(I0));
    ring.idx[slot] = ii;
}

template <int MODE, bool BELOW62>
__global__ void __launch_bounds__(kBlockThreads) abc_reject_kernel(const __grid_constant__ ModelParams p,
                                                                   const __grid_constant__ RejectArgs a)
{
    extern __shared__ int4 obs_s[];
    stage_observed(obs_s, a.obs, p.T);
    WarpRing* rings = reinterpret_cast<WarpRing*>(obs_s + (p.T + 1));
    const uint32_t lane = threadIdx.x & 31u;
    WarpRing& ring = rings[threadIdx.x >> 5];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int32_t T = p.T;

    bool active = false;
    uint64_t i = 0, acc = 0;
    // k: the next day pair of the lane's sample (1 with no sample); a sample's
    // simulated days, min(2 (k - 1), T), are counted when its lane takes the next
    uint32_t k = 1, days = 0;
    Theta t{};
    State x;
    uint32_t head = 0, tail = 0;     // ring entries consumed / produced (warp-uniform)
    bool exhausted = false;          // no indices left to claim (warp-uniform)

    while (true) {
        const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !active);
        const uint32_t need = __popc(idle);
        if (need >= kRefillMinIdle) {
            if (tail - head < need && !exhausted) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(a.next, 32ull);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (base >= a.n_samples) {
                    exhausted = true;
                } else {
                    const uint64_t left = a.n_samples - base;
                    const uint32_t made = left < 32 ? (uint32_t)left : 32u;
                    if (lane < made) {
                        const uint64_t ii = a.first_index + base + lane;
                        float th[8];
                        prior_draw(p, ii, th);
                        ring_put<MODE>(ring, (tail + lane) & (kRing - 1), p, ii, th, p.A0, p.room0);
                    }
                    tail += made;
                    if (made < 32 || base + 32 >= a.n_samples) exhausted = true;
                    __syncwarp();
                }
            }
            const uint32_t avail = tail - head;
            // every lane idle and nothing left to hand out (the indices are
            // exhausted: a claim would have refilled the ring otherwise); this
            // replaces a second ballot per day pair for the loop's exit
            if (need == 32 && avail == 0) break;
            if (!active) {
                const uint32_t rank = __popc(idle & lt_mask);
                if (rank < avail) {
                    const uint32_t slot = (head + rank) & (kRing - 1);
                    const float4 l = ring.lo[slot], h = ring.hi[slot];
                    i = ring.idx[slot];
                    t.a0 = l.x; t.a = l.y; t.n = l.z; t.beta = l.w;
                    t.gamma = h.x; t.delta = h.y; t.beta_eta = h.z;
                    x = state_from(__float_as_int(h.w), p.A0, p.R0, p.D0, p.room0);
                    days += min(2 * k - 2, (uint32_t)T);
                    acc = 0;
                    k = 1;
                    active = true;
                }
            }
            head += need < avail ? need : avail;
            __syncwarp();
        }

        // fast mode takes three day pairs per pass between hand-outs, cutting
        // the refill and accept checks; per 2^24 samples of P = 6e7, T = 100
        // (interleaved, three repeats): 1 pair 5.462 ms, 2 pairs 5.474, 3 pairs
        // 5.424, 4 pairs 5.438, 5 pairs 5.503. Exact mode's longer day ran
        // 13 % slower with two pairs.
        bool accept = false;
#pragma unroll
        for (int rep = 0; rep < ((MODE & kFast) ? 3 : 1); ++rep)
        if (active) {
            float z[10];
            day_pair_normals<MODE>(p, i, k, z);
            const int32_t d1 = (int32_t)(2 * k - 1);
            model_day<MODE>(x, t, p.inv_p, z);
            acc = BELOW62 ? add_day_sq_below62(acc, x, obs_s[d1]) : add_day_sq(acc, x, obs_s[d1]);
            if (d1 < T) {
                model_day<MODE>(x, t, p.inv_p, z + 5);
                acc = BELOW62 ? add_day_sq_below62(acc, x, obs_s[d1 + 1]) : add_day_sq(acc, x, obs_s[d1 + 1]);
            }
            const bool over = acc > a.acc_max;
            const bool last = d1 + 1 >= T;
            accept = !over && last;
            active = !(over || last);
            ++k;
        }
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, accept);
        if (mask) {
            const uint32_t leader = __ffs(mask) - 1;
            unsigned long long slot0 = 0;
            if (lane == leader) slot0 = atomicAdd(a.count, (unsigned long long)__popc(mask));
            slot0 = __shfl_sync(0xFFFFFFFFu, slot0, leader);
            if (accept) {
                const uint64_t slot = slot0 + __popc(mask & lt_mask);
                if (slot < a.capacity) {
                    float th[8];
                    prior_draw(p, i, th);
                    a.idx_out[slot] = i;
                    a.dist_out[slot] = __dsqrt_rn(__ull2double_rn(acc));
                    float4* to = reinterpret_cast<float4*>(a.theta_out + 8 * slot);
                    to[0] = make_float4(th[0], th[1], th[2], th[3]);
                    to[1] = make_float4(th[4], th[5], th[6], th[7]);
                }
            }
        }
    }
    // simulated model days of this warp (for throughput accounting), the
    // lane's last sample included
    days += min(2 * k - 2, (uint32_t)T);
    unsigned long long d = days;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, off);
    if (lane == 0 && a.sim_days) atomicAdd(a.sim_days, d);
}

// ---------------------------------------------------------------------------
// K2: every distance (and optionally every prior draw).
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kBlockThreads) abc_distance_kernel(const __grid_constant__ ModelParams p,
                                                                     const __grid_constant__ DistanceArgs a)
{
    extern __shared__ int4 obs_s[];
    stage_observed(obs_s, a.obs, p.T);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n_samples; j += stride) {
        const uint64_t i = a.first_index + j;
        float th[8];
        prior_draw(p, i, th);
        const Theta t = make_theta<MODE>(th, p.inv_p);
        const State x0 = init_state(t, p.A0, p.R0, p.D0, p.room0);
        const uint64_t acc = simulate_sample<MODE>(p, i, t, x0, obs_s, NoVisit());
        a.dist_out[j] = __dsqrt_rn(__ull2double_rn(acc));
        if (a.theta_out) {
            float4* to = reinterpret_cast<float4*>(a.theta_out + 8 * j);
            to[0] = make_float4(th[0], th[1], th[2], th[3]);
            to[1] = make_float4(th[4], th[5], th[6], th[7]);
        }
    }
}

// ---------------------------------------------------------------------------
// K3: trajectories of given (theta, sample index) pairs.
// ---------------------------------------------------------------------------
struct TrajVisit {
    int32_t* out;
    __device__ __forceinline__ void operator()(int32_t d, const State& x) const
    {
        int32_t* o = out + 6 * (size_t)d;
        o[0] = x.S; o[1] = x.I; o[2] = x.A; o[3] = x.R; o[4] = x.D; o[5] = x.Ru;
    }
};

template <int MODE>
__global__ void __launch_bounds__(kBlockThreads) abc_simulate_kernel(const __grid_constant__ ModelParams p,
                                                                     const __grid_constant__ SimulateArgs a)
{
    extern __shared__ int4 obs_s[];
    // no observed series here: a zero series keeps the distance code shared
    for (int32_t d = threadIdx.x; d <= p.T; d += blockDim.x) obs_s[d] = make_int4(0, 0, 0, 0);
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < a.B; b += stride) {
        float th[8];
        const float4* ti = reinterpret_cast<const float4*>(a.theta + 8 * b);
        const float4 t0 = ti[0], t1 = ti[1];
        th[0] = t0.x; th[1] = t0.y; th[2] = t0.z; th[3] = t0.w;
        th[4] = t1.x; th[5] = t1.y; th[6] = t1.z; th[7] = t1.w;
        const Theta t = make_theta<MODE>(th, p.inv_p);
        const State x0 = init_state(t, p.A0, p.R0, p.D0, p.room0);
        TrajVisit v{a.traj_out + (size_t)b * 6 * (size_t)(p.T + 1)};
        v(0, x0);
        simulate_sample<MODE>(p, a.sample_index[b], t, x0, obs_s, v);
    }
}

// ---------------------------------------------------------------------------
// K4: one day applied to given states.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kBlockThreads) abc_step_kernel(const __grid_constant__ ModelParams p,
                                                                 const __grid_constant__ StepArgs a)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < a.B; b += stride) {
        float th[8];
        for (int j = 0; j < 8; ++j) th[j] = a.theta[8 * b + j];
        const Theta t = make_theta<MODE>(th, p.inv_p);
        const int32_t* si = a.state_in + 6 * b;
        State x{si[0], si[1], si[2], si[3], si[4], si[5]};
        const int32_t d = a.day[b];
        float z[10];
        day_pair_normals<MODE>(p, a.sample_index[b], (uint32_t)(d + 1) >> 1, z);
        int32_t n[5];
        model_day<MODE>(x, t, p.inv_p, (d & 1) ? z : z + 5, n);
        int32_t* so = a.state_out + 6 * b;
        so[0] = x.S; so[1] = x.I; so[2] = x.A; so[3] = x.R; so[4] = x.D; so[5] = x.Ru;
        if (a.counts_out)
            for (int k = 0; k < 5; ++k) a.counts_out[5 * b + k] = n[k];
    }
}

// ---------------------------------------------------------------------------
// Quantile bands of trajectories: one block per (day, compartment) column,
// the B values sorted in shared memory by a bitonic network (padded to a power
// of two with INT_MAX), then order statistics floor(q (B - 1)).
// ---------------------------------------------------------------------------
constexpr int kBandThreads = 1024;
constexpr uint32_t kBandMaxB = 8192;   // the largest B the C ABI accepts (power of two)

__global__ void __launch_bounds__(kBandThreads) band_kernel(const int32_t* __restrict__ traj, uint32_t B, int32_t T,
                                                             const float* __restrict__ qpos, int32_t n_q,
                                                             float* __restrict__ bands)
{
    extern __shared__ int32_t v[];
    const int32_t d = blockIdx.x / 3, c = blockIdx.x % 3;
    uint32_t n2 = 1;
    while (n2 < B) n2 <<= 1;
    for (uint32_t b = threadIdx.x; b < n2; b += blockDim.x)
        v[b] = b < B ? traj[((size_t)b * (T + 1) + d) * 6 + 2 + c] : 0x7FFFFFFF;
    __syncthreads();
    // bitonic sort; each stage visits its n2 / 2 compare-exchange pairs
    // (i, i + j), i with bit j clear, rather than all n2 positions
    for (uint32_t k = 2; k <= n2; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t q = threadIdx.x; q < n2 / 2; q += blockDim.x) {
                const uint32_t i = ((q & ~(j - 1)) << 1) | (q & (j - 1)), p = i | j;
                const bool up = (i & k) == 0;
                const int32_t a = v[i], b2 = v[p];
                if ((a > b2) == up) {
                    v[i] = b2;
                    v[p] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int32_t k = threadIdx.x; k < n_q; k += blockDim.x) {
        const uint32_t r = (uint32_t)qpos[k];
        bands[((size_t)k * (T + 1) + d) * 3 + c] = (float)v[r];
    }
}

// ---------------------------------------------------------------------------
// Radix select of the k-th smallest distance: eight passes over the keys (the
// bit patterns of non-negative doubles order like the values), one 8-bit
// digit per pass from the top, one launch per pass. A pass histograms that
// digit among the keys whose higher digits equal the prefix chosen so far;
// the last block of the pass to finish (a ticket counter, after a memory
// fence) picks the digit holding the wanted rank and updates the state in
// device memory, so the passes run back to back with no host round trip. On
// the first pass (mask == 0) hist[256] counts the keys above +infinity's
// pattern: NaN and anything with the sign bit set (negative values and -0),
// which would not order like their values. hist[257] is the ticket counter.
// ---------------------------------------------------------------------------

// One warp: the digit of this pass is the first whose running count reaches
// the rank (k on the first pass); the rank becomes the rank within that
// digit's keys. Lane j holds bins 8j .. 8j + 7 in h (their sum in sum): a
// warp scan of the lanes' sums finds the lane, then that lane walks its eight
// bins and updates the state.
__device__ __forceinline__ void select_digit(const unsigned long long (&h)[8], unsigned long long sum,
                                             SelectState* st, int shift, uint64_t rank)
{
    const int lane = threadIdx.x & 31;
    // inclusive scan of the lanes' sums
    unsigned long long incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += v;
    }
    const uint32_t reach = __ballot_sync(0xFFFFFFFFu, incl >= rank);
    // the first lane whose running count reaches the rank (the last lane if
    // none does, which only invalid input allows)
    const int owner = reach ? __ffs(reach) - 1 : 31;
    if (lane == owner) {
        uint64_t below = incl - sum;
        int i = 0;
        for (; i < 7; ++i) {
            if (below + h[i] >= rank) break;
            below += h[i];
        }
        st->rank = rank - below;
        st->prefix |= (uint64_t)(8 * lane + i) << shift;
        st->mask |= (uint64_t)0xFF << shift;
    }
}

__global__ void __launch_bounds__(kBlockThreads) digit_pass_kernel(const double* __restrict__ dist, uint64_t n,
                                                                   SelectState* __restrict__ st, int shift,
                                                                   uint64_t k, unsigned long long* __restrict__ hist)
{
    __shared__ unsigned int h[257];
    __shared__ bool last;
    for (int b = threadIdx.x; b < 257; b += blockDim.x) h[b] = 0;
    // the previous pass (or the kernel that wrote the distances) completes
    // before the state and the keys are read; the next pass may launch now
    griddep_wait();
    griddep_release();
    __syncthreads();
    const uint64_t prefix = st->prefix, prefix_mask = st->mask;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const bool first = prefix_mask == 0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint64_t key = (uint64_t)__double_as_longlong(dist[j]);
        if ((key & prefix_mask) == prefix) atomicAdd(&h[(key >> shift) & 0xFFu], 1u);
        if (first && key > 0x7FF0000000000000ull) atomicAdd(&h[256], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 257; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], (unsigned long long)h[b]);
    // the block's counts are in before its ticket is taken
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&hist[257], 1ull) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    // the last block: every block's counts are in; read them past L1
    __threadfence();
    const int lane = threadIdx.x;
    unsigned long long hb[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        hb[i] = __ldcg(&hist[8 * lane + i]);
        sum += hb[i];
    }
    const uint64_t rank = first ? k : st->rank;
    if (first && lane == 0) st->bad = __ldcg(&hist[256]);
    __syncwarp();
    // the histogram and the ticket counter zeroed for the next pass
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[8 * lane + i] = 0;
    if (lane == 0) {
        hist[256] = 0;
        hist[257] = 0;
    }
    select_digit(hb, sum, st, shift, rank);
}

// ---------------------------------------------------------------------------
// Samples accepted at eps from distances already computed (Sec. 2.2: accept
// when the distance is at most eps): sample j is accepted iff dist[j] <= eps.
// Each warp takes 32 consecutive samples at a time, reserves the slots of its
// accepts with one atomicAdd and writes index, distance and theta. Every
// accept is counted; only slots below capacity are written.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockThreads) select_below_kernel(const __grid_constant__ SelectArgs a)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    griddep_wait();   // the distances and the selected key are complete
    const double eps = a.eps_key ? __longlong_as_double((long long)a.eps_key->prefix) : a.eps;
    for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32; base < a.n;
         base += warps * 32) {
        const uint64_t j = base + lane;
        const bool take = j < a.n && a.dist[j] <= eps;
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, take);
        if (!mask) continue;
        unsigned long long slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(a.count, (unsigned long long)__popc(mask));
        slot0 = __shfl_sync(0xFFFFFFFFu, slot0, 0);
        if (!take) continue;
        const uint64_t slot = slot0 + __popc(mask & ((1u << lane) - 1u));
        if (slot >= a.capacity) continue;
        a.idx_out[slot] = a.first_index + j;
        a.dist_out[slot] = a.dist[j];
        if (a.theta_out) {
            const float4* src = reinterpret_cast<const float4*>(a.theta + 8 * j);
            float4* to = reinterpret_cast<float4*>(a.theta_out + 8 * slot);
            to[0] = src[0];
            to[1] = src[1];
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Resident blocks per SM times the SM count, for a kernel, dynamic shared
// memory size and device; looked up once and cached (the launch path then
// makes no occupancy query). The kernel's dynamic shared-memory limit is one
// value per kernel and device: it is only ever raised, to the largest size
// launched so far, so a call with a shorter horizon never lowers it below
// what a cached longer one needs.
template <typename K>
static cudaError_t grid_for(K kernel, size_t smem, int* grid)
{
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> cache;
    static std::map<std::pair<const void*, int>, size_t> limit;   // largest limit set per kernel and device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > 48 * 1024) {
        size_t& lim = limit[std::make_pair((const void*)kernel, dev)];
        if (lim < smem) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            lim = smem;
        }
    }
    const auto key = std::make_tuple((const void*)kernel, dev, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *grid = it->second;
        return cudaSuccess;
    }
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlockThreads, smem);
    if (e != cudaSuccess) return e;
    *grid = sms * (per_sm > 0 ? per_sm : 1);
    cache[key] = *grid;
    return cudaSuccess;
}

static int blocks_for(uint64_t n, int cap)
{
    const uint64_t b = (n + kBlockThreads - 1) / kBlockThreads;
    return (int)(b < (uint64_t)cap ? (b > 0 ? b : 1) : (uint64_t)cap);
}

size_t reject_smem_bytes(int32_t T) { return sizeof(int4) * (size_t)(T + 1) + sizeof(WarpRing) * kWarpsPerBlock; }

template <int MODE, bool BELOW62>
static cudaError_t launch_reject_t(const ModelParams& p, const RejectArgs& a, cudaStream_t s, int* blocks_out)
{
    const size_t smem = reject_smem_bytes(p.T);
    int grid = 0;
    cudaError_t e = grid_for(abc_reject_kernel<MODE, BELOW62>, smem, &grid);
    if (e != cudaSuccess) return e;
    // persistent: every resident block loops over claimed index chunks
    const uint64_t chunks = (a.n_samples + 31) / 32;
    const uint64_t want = (chunks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (want < (uint64_t)grid) grid = (int)(want > 0 ? want : 1);
    if (blocks_out) *blocks_out = grid;
    abc_reject_kernel<MODE, BELOW62><<<grid, kBlockThreads, smem, s>>>(p, a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_reject_m(const ModelParams& p, const RejectArgs& a, cudaStream_t s, int* blocks_out)
{
    const bool below62 = a.acc_max < 0x4000000000000000ull;
    return below62 ? launch_reject_t<MODE, true>(p, a, s, blocks_out) : launch_reject_t<MODE, false>(p, a, s, blocks_out);
}

#define ABC_MODE_DISPATCH(fn, mode, ...)                        \
    ((mode) == kFast ? fn<kFast>(__VA_ARGS__)                   \
     : (mode) == kExact ? fn<kExact>(__VA_ARGS__)               \
     : (mode) == (kFast | kLiteral) ? fn<kFast | kLiteral>(__VA_ARGS__) \
                                  : fn<kExact | kLiteral>(__VA_ARGS__))

cudaError_t launch_reject(const ModelParams& p, const RejectArgs& a, int mode, cudaStream_t s, int* blocks_out)
{
    return ABC_MODE_DISPATCH(launch_reject_m, mode, p, a, s, blocks_out);
}

template <int MODE>
static cudaError_t launch_distances_m(const ModelParams& p, const DistanceArgs& a, cudaStream_t s)
{
    const size_t smem = sizeof(int4) * (size_t)(p.T + 1);
    int grid = 0;
    cudaError_t e = grid_for(abc_distance_kernel<MODE>, smem, &grid);
    if (e != cudaSuccess) return e;
    grid = blocks_for(a.n_samples, grid);
    abc_distance_kernel<MODE><<<grid, kBlockThreads, smem, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_distances(const ModelParams& p, const DistanceArgs& a, int mode, cudaStream_t s)
{
    return ABC_MODE_DISPATCH(launch_distances_m, mode, p, a, s);
}

template <int MODE>
static cudaError_t launch_simulate_m(const ModelParams& p, const SimulateArgs& a, cudaStream_t s)
{
    const size_t smem = sizeof(int4) * (size_t)(p.T + 1);
    int grid = 0;
    cudaError_t e = grid_for(abc_simulate_kernel<MODE>, smem, &grid);
    if (e != cudaSuccess) return e;
    grid = blocks_for(a.B, grid);
    abc_simulate_kernel<MODE><<<grid, kBlockThreads, smem, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_simulate(const ModelParams& p, const SimulateArgs& a, int mode, cudaStream_t s)
{
    return ABC_MODE_DISPATCH(launch_simulate_m, mode, p, a, s);
}

template <int MODE>
static cudaError_t launch_step_m(const ModelParams& p, const StepArgs& a, cudaStream_t s)
{
    int grid = 0;
    cudaError_t e = grid_for(abc_step_kernel<MODE>, 0, &grid);
    if (e != cudaSuccess) return e;
    grid = blocks_for(a.B, grid);
    abc_step_kernel<MODE><<<grid, kBlockThreads, 0, s>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_step(const ModelParams& p, const StepArgs& a, int mode, cudaStream_t s)
{
    return ABC_MODE_DISPATCH(launch_step_m, mode, p, a, s);
}

cudaError_t launch_bands(const int32_t* traj, uint32_t B, int32_t T, const float* qpos, int32_t n_q, float* bands,
                         cudaStream_t s)
{
    if (B < 1 || B > kBandMaxB) return cudaErrorInvalidValue;
    uint32_t n2 = 1;
    while (n2 < B) n2 <<= 1;
    const size_t smem = sizeof(int32_t) * n2;
    if (smem > 48 * 1024) {
        // set once per device to the largest size B <= ABC_PROJECT_MAX_B can need
        static std::mutex mu;
        static std::map<int, bool> done;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        if (!done[dev]) {
            e = cudaFuncSetAttribute(band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(int32_t) * kBandMaxB));
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    band_kernel<<<3 * (T + 1), kBandThreads, smem, s>>>(traj, B, T, qpos, n_q, bands);
    return cudaGetLastError();
}

cudaError_t launch_select_below(const SelectArgs& a, cudaStream_t s)
{
    int grid = 0;
    cudaError_t e = grid_for(select_below_kernel, 0, &grid);
    if (e != cudaSuccess) return e;
    grid = blocks_for(a.n, grid);
    e = launch_overlapped(select_below_kernel, dim3(grid), dim3(kBlockThreads), 0, s, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_kth_select(const double* dist, uint64_t n, uint64_t k, unsigned long long* hist, SelectState* st,
                              cudaStream_t s)
{
    int grid = 0;
    cudaError_t e = grid_for(digit_pass_kernel, 0, &grid);
    if (e != cudaSuccess) return e;
    grid = blocks_for(n, grid);
    for (int shift = 56; shift >= 0 && e == cudaSuccess; shift -= 8)
        e = launch_overlapped(digit_pass_kernel, dim3(grid), dim3(kBlockThreads), 0, s, dist, n, st, shift, k, hist);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace abcgb
