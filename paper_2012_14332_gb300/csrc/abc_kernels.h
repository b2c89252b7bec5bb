// abc_kernels.h -- internal launch interface between the C ABI (abc_api.cu) and
// the kernels (abc_kernels.cu). Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace abcgb {

constexpr int kBlockThreads = 256;

// Programmatic dependent launch: a kernel launched with launch_overlapped may
// start before the previous kernel in its stream has finished. griddep_wait
// returns once that kernel has completed and its memory is visible (at once
// for a plain launch); griddep_release lets the next overlapped launch start
// once every CTA of this kernel has released or exited.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// A launch with programmatic stream serialization: the kernel must call
// griddep_wait before it touches anything the previous kernel writes or
// reads.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_overlapped(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

struct ModelParams;

struct RejectArgs {
    const int4* obs;              // device [T+1] (A, R, D, 0)
    uint64_t first_index, n_samples;
    uint64_t acc_max;             // accept iff distance^2 <= acc_max
    unsigned long long* count;    // device counter of accepts, zeroed before launch
    unsigned long long* next;     // device counter of claimed indices, zeroed before launch
    unsigned long long* sim_days; // device counter of simulated days (zeroed) or null
    uint64_t capacity;
    float* theta_out;             // device [capacity][8]
    double* dist_out;             // device [capacity]
    uint64_t* idx_out;            // device [capacity]
};

struct DistanceArgs {
    const int4* obs;
    uint64_t first_index, n_samples;
    double* dist_out;             // device [n_samples]
    float* theta_out;             // device [n_samples][8] or null
};

struct SimulateArgs {
    const float* theta;           // device [B][8]
    const uint64_t* sample_index; // device [B]
    uint64_t B;
    int32_t* traj_out;            // device [B][T+1][6]
};

struct StepArgs {
    const float* theta;           // device [B][8]
    const int32_t* state_in;      // device [B][6]
    const uint64_t* sample_index; // device [B]
    const int32_t* day;           // device [B]
    uint64_t B;
    int32_t* state_out;           // device [B][6]
    int32_t* counts_out;          // device [B][5] or null
};

// One region of a batched launch (device-resident table; see abc_batch.cu).
constexpr int kMaxRegions = 32;
struct RegionDev {
    uint64_t first_index;          // first sample index of the current run (advanced after each run)
    uint64_t n_samples;            // samples per run
    uint64_t chunk_begin;          // first 32-sample chunk of this region in the run's chunk space
    uint64_t acc_max;              // accept iff distance^2 <= acc_max
    uint64_t capacity;             // accepted samples kept
    float* theta_out;              // device [capacity][8]
    double* dist_out;              // device [capacity]
    uint64_t* idx_out;             // device [capacity]
    const float* theta_in;         // device [n_samples][8] proposals, or null: prior draws
    unsigned long long* counters;  // device [2]: accepted, simulated days
    int32_t T, P, room0, A0, R0, D0;
    uint32_t ctr3_base;            // 4 * stream
    float inv_p;
    uint32_t obs_off;              // first day of this region in the concatenated observed series
    uint32_t pad_;
};

struct BatchArgs {
    const RegionDev* regions;      // device [n_regions]
    int32_t n_regions;
    uint64_t total_chunks;
    const int4* obs;               // device, concatenated (A, R, D, 0) per day of every region
    int32_t n_obs_smem;            // > 0: all n_obs_smem entries of obs are staged in shared memory
    unsigned long long* next;      // claimed chunks, zeroed before each run
};

// The batched kernel stages every region's observed series in shared memory
// when together they hold at most this many days (32 KB), and reads them
// through the read-only data cache otherwise.
constexpr int32_t kBatchObsSmemMax = 2048;

// Launch shapes the batched kernel is compiled for (the autotuner's space).
struct BatchShape {
    int block_threads;   // 128, 256 or 512
    int pairs;           // day pairs per loop iteration (1 or 2)
    int blocks_per_sm;   // resident blocks requested per SM (0 = as many as fit)
    int lean;            // 1: region constants read from shared memory (fast mode, 256 threads)
};
int batch_shape_count();
BatchShape batch_shape(int index);
bool batch_shape_supported(const BatchShape& shape, bool fast);   // the lean form is fast mode only

// below62: every region's acc_max < 2^62 (the cheaper distance accumulation)
cudaError_t launch_batch(const ModelParams& p, const BatchArgs& a, bool fast, bool below62, const BatchShape& shape,
                         cudaStream_t s);
cudaError_t launch_advance(RegionDev* regions, int32_t n_regions, cudaStream_t s);
cudaError_t prepare_batch(bool fast, bool below62, int32_t n_obs_smem, const BatchShape& shape);

size_t reject_smem_bytes(int32_t T);
// mode: kExact or kFast, optionally | kLiteral (see abc_model.cuh)
cudaError_t launch_reject(const ModelParams& p, const RejectArgs& a, int mode, cudaStream_t s, int* blocks_out);
cudaError_t launch_distances(const ModelParams& p, const DistanceArgs& a, int mode, cudaStream_t s);
cudaError_t launch_simulate(const ModelParams& p, const SimulateArgs& a, int mode, cudaStream_t s);
cudaError_t launch_step(const ModelParams& p, const StepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_bands(const int32_t* traj, uint32_t B, int32_t T, const float* qpos, int32_t n_q, float* bands,
                         cudaStream_t s);
// Radix select of the k-th smallest of n distances, all passes on the device:
// hist (258 counters: the histogram and a ticket counter) and st zeroed by the
// caller, and left zeroed and holding the result; afterwards st->prefix is
// the k-th smallest key and st->bad the number of invalid keys (NaN, sign bit
// set), in which case the prefix is meaningless.
struct SelectState {
    unsigned long long prefix, mask, rank, bad;
};
// Compaction of the samples with dist[j] <= eps (theta, theta_out may both be
// NULL); *count (zeroed by the caller) receives the number of accepts. With
// eps_key set, eps is the value whose bit pattern is eps_key->prefix (the
// radix select's k-th smallest, computed on the device) instead of `eps`.
struct SelectArgs {
    const double* dist;
    const float* theta;
    uint64_t n, first_index;
    double eps;
    const SelectState* eps_key;
    float* theta_out;
    double* dist_out;
    uint64_t* idx_out;
    uint64_t capacity;
    unsigned long long* count;
};
cudaError_t launch_select_below(const SelectArgs& a, cudaStream_t s);
cudaError_t launch_kth_select(const double* dist, uint64_t n, uint64_t k, unsigned long long* hist, SelectState* st,
                              cudaStream_t s);

}  // namespace abcgb
