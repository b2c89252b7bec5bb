// abc_batch.cu -- batched ABC rejection over a table of regions in one
// persistent launch (many regions with their own population, horizon T,
// tolerance eps, observed series, random stream and sample range).
//
// Same per-sample method and early rejection as abc_reject_kernel (paper
// Sec. 2.1, 2.2, 3.1); what changes is where a lane's constants come from:
// each 32-sample chunk belongs to one region, and a lane that takes a sample
// also takes its region's T, eps threshold, stream, 1/P and observed-series
// offset from the region table staged in shared memory. The observed series
// are staged in shared memory too when all regions' series fit (OBS_S), and
// read through the read-only data cache otherwise. Chunks are claimed from
// one counter across all regions, so
// uneven regions balance across the whole GPU. Accepted samples go to their
// region's buffers (one atomicAdd per accept: accepts are rare).
#include <cstdint>
#include <cuda_runtime.h>

#include "abc_kernels.h"
#include "abc_model.cuh"

namespace abcgb {

namespace {

constexpr int kRingB = 64;
// idle lanes get new samples once at least this many are idle, as in
// abc_reject_kernel (all 32 always qualify)
constexpr uint32_t kRefillMinIdleB = 2;

// A ring entry holds the sample's parameters as the day loop uses them and its
// initial I0 (worked out when the ring is refilled, one sample per lane), so
// handing a sample to an idle lane is a few shared-memory reads.
struct BatchRing {
    float4 lo[kRingB];      // Theta a0, a, n, beta
    float4 hi[kRingB];      // Theta gamma, delta, beta_eta; I0 (int32 bits)
    uint64_t idx[kRingB];
    int32_t region[kRingB];
};

__device__ __forceinline__ void load_theta(const float* src, float th[8])
{
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4 l = __ldg(s4), h = __ldg(s4 + 1);
    th[0] = l.x; th[1] = l.y; th[2] = l.z; th[3] = l.w;
    th[4] = h.x; th[5] = h.y; th[6] = h.z; th[7] = h.w;
}

// Region constants a lane keeps in registers for its current sample.
struct LaneRegion {
    int32_t r, T;
    uint32_t ctr3, obs_off;
    uint64_t acc_max;
    float inv_p;
};

// BELOW62: every region's acc_max < 2^62, so the running sum can be clamped at
// 2^62 each day instead of saturating exactly at 2^63 (fewer instructions; the
// accept sets and accepted distances are the same, as in abc_reject_kernel).
//
// LEAN: a lane keeps only its region's index and reads the region's constants
// from the shared table where it uses them; this fits 64 registers (four
// 256-thread blocks per SM instead of three) for a few shared-memory reads per
// day pair. A lane adds its samples' simulated days in a 32-bit register and
// moves them to the block's 64-bit per-region count when its region changes
// (chunks are laid out region by region, so rarely) or the register passes
// 2^31, and at the end. Adding each sample's days to the shared count with a
// 64-bit shared-memory atomic cost 5 % of the 16-region stream (52.5 -> 49.7
// ms) and 3 % of the three-region workload. The autotuner chooses between the
// two forms; with the register count it takes the lean form on both
// workloads (16-region stream 49.1 ms, three-region workload 2.12 ms, against
// 56.4 and 2.18 ms for the standard form).
template <int MODE, int BLOCK, int PAIRS, bool BELOW62, bool OBS_S, bool LEAN>
__global__ void __launch_bounds__(BLOCK, LEAN ? 4 : 1) abc_batch_kernel(const __grid_constant__ ModelParams p,
                                                          const __grid_constant__ BatchArgs a)
{
    __shared__ RegionDev reg_s[kMaxRegions];
    __shared__ unsigned long long days_s[LEAN ? kMaxRegions : 1];   // LEAN: simulated days per region
    extern __shared__ BatchRing rings[];   // one per warp, then (OBS_S) the observed series
    int4* obs_s = reinterpret_cast<int4*>(rings + BLOCK / 32);
    for (int r = threadIdx.x; r < a.n_regions; r += BLOCK) {
        reg_s[r] = a.regions[r];
        if (LEAN) days_s[r] = 0;
    }
    if (OBS_S)
        for (int q = threadIdx.x; q < a.n_obs_smem; q += BLOCK) obs_s[q] = a.obs[q];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    BatchRing& ring = rings[threadIdx.x >> 5];
    const uint32_t lt_mask = (1u << lane) - 1u;

    bool active = false;
    uint64_t i = 0, acc = 0;
    // k: the next day pair of the lane's sample (1 with no sample); a sample's
    // simulated days, min(2 (k - 1), T), are counted when its lane takes the next
    uint32_t k = 1;
    Theta t{};
    State x;
    LaneRegion lr{0, 1, 0, 0, 0, 0.0f};
    int32_t days_region = -1;
    unsigned long long days = 0;
    uint32_t days32 = 0;   // LEAN: days of the lane's samples in region lr.r not yet added
    uint32_t head = 0, tail = 0;
    bool exhausted = false;
    // Chunks are claimed one refill ahead (lane 0 holds the claim), so the
    // atomic's round trip overlaps the day pairs simulated before the next
    // refill; a claim made is always consumed by this warp. Measured: 16-region
    // stream 58.2 -> 56.8 ms, config 3 2.317 -> 2.289 ms (the single-region
    // kernel, whose samples run longer between refills, gains nothing).
    unsigned long long claim = 0;
    if (lane == 0) claim = atomicAdd(a.next, 1ull);
    // region of the warp's last claim: a warp's claims only grow and regions
    // occupy consecutive chunk ranges, so the region index only moves forward
    int32_t claim_r = 0;

    while (true) {
        const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !active);
        const uint32_t need = __popc(idle);
        if (need >= kRefillMinIdleB) {
            if (tail - head < need && !exhausted) {
                const unsigned long long c = __shfl_sync(0xFFFFFFFFu, claim, 0);
                if (c >= a.total_chunks) {
                    exhausted = true;
                } else {
                    if (lane == 0) claim = atomicAdd(a.next, 1ull);
                    int32_t r = claim_r;
                    while (r + 1 < a.n_regions && reg_s[r + 1].chunk_begin <= c) ++r;
                    claim_r = r;
                    const RegionDev& R = reg_s[r];
                    const uint64_t j0 = (c - R.chunk_begin) * 32;
                    const uint64_t left = R.n_samples - j0;
                    const uint32_t made = left < 32 ? (uint32_t)left : 32u;
                    float th[8];
                    bool keep = false;
                    if (lane < made) {
                        if (R.theta_in)
                            load_theta(R.theta_in + 8 * (j0 + lane), th);
                        else
                            prior_draw_s(p, R.first_index + j0 + lane, R.ctr3_base, th);
                        // a proposal whose first coordinate is NaN is skipped (no simulation)
                        keep = th[0] == th[0];
                    }
                    const uint32_t kept = __ballot_sync(0xFFFFFFFFu, keep);
                    if (keep) {
                        const uint32_t slot = (tail + __popc(kept & lt_mask)) & (kRingB - 1);
                        const Theta tt = make_theta<MODE>(th, R.inv_p);
                        const int32_t I0 = initial_infected(tt, R.A0, R.room0);
                        ring.lo[slot] = make_float4(tt.a0, tt.a, tt.n, tt.beta);
                        ring.hi[slot] = make_float4(tt.gamma, tt.delta, tt.beta_eta, __int_as_float(I0));
                        ring.idx[slot] = R.first_index + j0 + lane;
                        ring.region[slot] = r;
                    }
                    tail += __popc(kept);
                    __syncwarp();
                }
            }
            const uint32_t avail = tail - head;
            // every lane idle and nothing left to hand out: the chunks are
            // exhausted (a claim adds at least one entry otherwise, since a
            // chunk of only skipped proposals is followed by another claim)
            if (need == 32 && avail == 0 && exhausted) break;
            if (!active) {
                const uint32_t rank = __popc(idle & lt_mask);
                if (rank < avail) {
                    const uint32_t slot = (head + rank) & (kRingB - 1);
                    const float4 l = ring.lo[slot], h = ring.hi[slot];
                    i = ring.idx[slot];
                    const int32_t r = ring.region[slot];
                    const RegionDev& R = reg_s[r];
                    // the days of the lane's previous sample (k = 1: none)
                    if (LEAN) {
                        days32 += min(2 * k - 2, (uint32_t)reg_s[lr.r].T);
                        if (r != lr.r || days32 >= 0x80000000u) {
                            if (days32) atomicAdd(&days_s[lr.r], (unsigned long long)days32);
                            days32 = 0;
                        }
                    } else {
                        days += min(2 * k - 2, (uint32_t)lr.T);
                    }
                    lr.r = r;
                    if (!LEAN) {
                        if (r != days_region) {
                            if (days_region >= 0 && days) atomicAdd(reg_s[days_region].counters + 1, days);
                            days = 0;
                            days_region = r;
                        }
                        lr.T = R.T;
                        lr.ctr3 = R.ctr3_base;
                        lr.obs_off = R.obs_off;
                        lr.acc_max = R.acc_max;
                        lr.inv_p = R.inv_p;
                    }
                    t.a0 = l.x; t.a = l.y; t.n = l.z; t.beta = l.w;
                    t.gamma = h.x; t.delta = h.y; t.beta_eta = h.z;
                    x = state_from(__float_as_int(h.w), R.A0, R.R0, R.D0, R.room0);
                    acc = 0;
                    k = 1;
                    active = true;
                }
            }
            head += need < avail ? need : avail;
            __syncwarp();
        }

        bool accept = false;
#pragma unroll
        for (int rep = 0; rep < PAIRS; ++rep) {
            if (active) {
                const RegionDev& R = reg_s[lr.r];
                float z[10];
                day_pair_normals_s<MODE>(p, i, k, LEAN ? R.ctr3_base : lr.ctr3, z);
                const int32_t d1 = (int32_t)(2 * k - 1);
                const int4* obs = (OBS_S ? obs_s : a.obs) + (LEAN ? R.obs_off : lr.obs_off);
                // fast mode folds 1/P into theta at the hand-out; only exact mode reads it per day
                const float inv_p = is_fast(MODE) ? 0.0f : (LEAN ? R.inv_p : lr.inv_p);
                model_day<MODE>(x, t, inv_p, z);
                const int4 o1 = OBS_S ? obs[d1] : __ldg(obs + d1);
                acc = BELOW62 ? add_day_sq_below62(acc, x, o1) : add_day_sq(acc, x, o1);
                const int32_t T = LEAN ? R.T : lr.T;
                if (d1 < T) {
                    model_day<MODE>(x, t, inv_p, z + 5);
                    const int4 o2 = OBS_S ? obs[d1 + 1] : __ldg(obs + d1 + 1);
                    acc = BELOW62 ? add_day_sq_below62(acc, x, o2) : add_day_sq(acc, x, o2);
                }
                const bool over = acc > (LEAN ? R.acc_max : lr.acc_max);
                const bool last = d1 + 1 >= T;
                accept = !over && last;
                active = !(over || last);
                ++k;
            }
        }
        if (accept) {
            const RegionDev& R = reg_s[lr.r];
            const unsigned long long slot = atomicAdd(R.counters, 1ull);
            if (slot < R.capacity) {
                float th[8];
                if (R.theta_in)
                    load_theta(R.theta_in + 8 * (i - R.first_index), th);
                else
                    prior_draw_s(p, i, R.ctr3_base, th);
                R.idx_out[slot] = i;
                R.dist_out[slot] = __dsqrt_rn(__ull2double_rn(acc));
                float4* to = reinterpret_cast<float4*>(R.theta_out + 8 * slot);
                to[0] = make_float4(th[0], th[1], th[2], th[3]);
                to[1] = make_float4(th[4], th[5], th[6], th[7]);
            }
        }
    }
    // the days of each lane's last sample
    if (LEAN) {
        days32 += min(2 * k - 2, (uint32_t)reg_s[lr.r].T);
        if (days32) atomicAdd(&days_s[lr.r], (unsigned long long)days32);
        __syncthreads();
        for (int r = threadIdx.x; r < a.n_regions; r += BLOCK)
            if (days_s[r]) atomicAdd(reg_s[r].counters + 1, days_s[r]);
    } else {
        days += min(2 * k - 2, (uint32_t)lr.T);
        if (days_region >= 0 && days) atomicAdd(reg_s[days_region].counters + 1, days);
    }
}

__global__ void advance_kernel(RegionDev* regions, int32_t n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) regions[r].first_index += regions[r].n_samples;
}

}  // namespace

static const BatchShape kShapes[] = {
    {256, 1, 0, 0}, {128, 1, 0, 0}, {512, 1, 0, 0}, {256, 2, 0, 0}, {128, 2, 0, 0}, {512, 2, 0, 0},
    {256, 1, 2, 0}, {256, 1, 3, 0}, {256, 1, 0, 1}, {256, 2, 0, 1},
};

int batch_shape_count() { return (int)(sizeof kShapes / sizeof kShapes[0]); }
BatchShape batch_shape(int index) { return kShapes[index]; }
bool batch_shape_supported(const BatchShape& shape, bool fast) { return fast || !shape.lean; }

// With a == NULL only prepares: sets the kernel's dynamic shared-memory limit
// (the rings, and the observed series with OBS_S) and resolves its occupancy,
// so that a launch, or a graph capture of one, makes no attribute calls.
template <int MODE, int BLOCK, int PAIRS, bool BELOW62, bool OBS_S, bool LEAN = false>
static cudaError_t launch_t(const ModelParams& p, const BatchArgs* a, int32_t n_obs_smem, int blocks_per_sm,
                            cudaStream_t s)
{
    auto kernel = abc_batch_kernel<MODE, BLOCK, PAIRS, BELOW62, OBS_S, LEAN>;
    const size_t smem = sizeof(BatchRing) * (BLOCK / 32) + (OBS_S ? sizeof(int4) * (size_t)n_obs_smem : 0);
    int dev = 0, sms = 0, fit = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (!a) {
        // the limit is the kernel's, shared by every plan: set the largest
        // this instantiation can need, so no plan lowers another's
        const size_t most = sizeof(BatchRing) * (BLOCK / 32) + (OBS_S ? sizeof(int4) * (size_t)kBatchObsSmemMax : 0);
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, BLOCK, smem);
    if (e != cudaSuccess) return e;
    if (fit < 1) fit = 1;
    const int per_sm = (blocks_per_sm > 0 && blocks_per_sm < fit) ? blocks_per_sm : fit;
    if (!a) return cudaSuccess;
    uint64_t want = (a->total_chunks + BLOCK / 32 - 1) / (BLOCK / 32);
    int grid = sms * per_sm;
    if (want < (uint64_t)grid) grid = (int)(want > 0 ? want : 1);
    kernel<<<grid, BLOCK, smem, s>>>(p, *a);
    return cudaGetLastError();
}

template <int MODE, bool B62, bool OS>
static cudaError_t dispatch(const ModelParams& p, const BatchArgs* a, int32_t n_obs_smem, const BatchShape& sh,
                            cudaStream_t s)
{
    const int bps = sh.blocks_per_sm;
    // the lean form is compiled for fast mode at 256 threads, where it raises occupancy
    if (sh.lean) {
        if constexpr (MODE == kFast) {
            if (sh.block_threads == 256 && sh.pairs == 1) return launch_t<MODE, 256, 1, B62, OS, true>(p, a, n_obs_smem, bps, s);
            if (sh.block_threads == 256 && sh.pairs == 2) return launch_t<MODE, 256, 2, B62, OS, true>(p, a, n_obs_smem, bps, s);
        }
        return cudaErrorInvalidValue;
    }
    if (sh.block_threads == 128 && sh.pairs == 1) return launch_t<MODE, 128, 1, B62, OS>(p, a, n_obs_smem, bps, s);
    if (sh.block_threads == 256 && sh.pairs == 1) return launch_t<MODE, 256, 1, B62, OS>(p, a, n_obs_smem, bps, s);
    if (sh.block_threads == 512 && sh.pairs == 1) return launch_t<MODE, 512, 1, B62, OS>(p, a, n_obs_smem, bps, s);
    if (sh.block_threads == 128 && sh.pairs == 2) return launch_t<MODE, 128, 2, B62, OS>(p, a, n_obs_smem, bps, s);
    if (sh.block_threads == 256 && sh.pairs == 2) return launch_t<MODE, 256, 2, B62, OS>(p, a, n_obs_smem, bps, s);
    if (sh.block_threads == 512 && sh.pairs == 2) return launch_t<MODE, 512, 2, B62, OS>(p, a, n_obs_smem, bps, s);
    return cudaErrorInvalidValue;
}

template <bool B62, bool OS>
static cudaError_t dispatch_mode(const ModelParams& p, const BatchArgs* a, bool fast, int32_t n_obs_smem,
                                 const BatchShape& sh, cudaStream_t s)
{
    return fast ? dispatch<kFast, B62, OS>(p, a, n_obs_smem, sh, s) : dispatch<kExact, B62, OS>(p, a, n_obs_smem, sh, s);
}

static cudaError_t dispatch_all(const ModelParams& p, const BatchArgs* a, bool fast, bool below62, int32_t n_obs_smem,
                                const BatchShape& sh, cudaStream_t s)
{
    if (n_obs_smem < 0 || n_obs_smem > kBatchObsSmemMax) return cudaErrorInvalidValue;
    if (n_obs_smem > 0)
        return below62 ? dispatch_mode<true, true>(p, a, fast, n_obs_smem, sh, s)
                       : dispatch_mode<false, true>(p, a, fast, n_obs_smem, sh, s);
    return below62 ? dispatch_mode<true, false>(p, a, fast, 0, sh, s) : dispatch_mode<false, false>(p, a, fast, 0, sh, s);
}

cudaError_t launch_batch(const ModelParams& p, const BatchArgs& a, bool fast, bool below62, const BatchShape& shape,
                         cudaStream_t s)
{
    return dispatch_all(p, &a, fast, below62, a.n_obs_smem, shape, s);
}

cudaError_t prepare_batch(bool fast, bool below62, int32_t n_obs_smem, const BatchShape& shape)
{
    ModelParams p{};
    return dispatch_all(p, nullptr, fast, below62, n_obs_smem, shape, nullptr);
}

cudaError_t launch_advance(RegionDev* regions, int32_t n_regions, cudaStream_t s)
{
    advance_kernel<<<1, 32, 0, s>>>(regions, n_regions);
    return cudaGetLastError();
}

}  // namespace abcgb
