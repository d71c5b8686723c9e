// Argument block of the rollout kernel and the launch entry points of the rollout code.
#pragma once

#include "vpm_device.cuh"

namespace vpm {

struct RolloutArgs {
    DevParams p;
    const void *root_part;      // float4 or Part64 records
    const int *root_n;
    const double *root_glider;  // 7
    const double *root_hist;    // n_b + 2
    long long root_stride;      // records between rollouts of the root arrays (0: shared root)
    long long state_stride;     // doubles between rollouts of glider / hist arrays (0: shared)
    int H, K, cap, step0;
    const float *controls;      // K x ctrl_stride (null: u_const every step)
    int ctrl_stride;
    double u_const;
    int rid0;                   // index of the first rollout of this launch
    float *costs;
    double *final_glider, *traj, *field;
    int field_cap;
    int *count;
    // write-back of the state (vpm_step, per-launch form)
    long long out_stride;       // records between rollouts of the output arrays
    long long out_state_stride; // doubles between rollouts of the output glider / hist arrays
    void *out_part;
    int *out_n;
    double *out_glider, *out_hist;
    // single-step probes
    double *probe_fm, *probe_gs, *probe_vel, *probe_vt;
    int *status;
    // persistent uneven batches: per-rollout record offsets into root_part (overrides
    // root_stride), the order in which rollouts are claimed, and the claim counter
    const long long *root_offset;
    const int *order;
    int *counter;
    int n_items;
    // per-rollout initial glider states (K x 7, overrides root_glider; null: the root's)
    const double *x0;
    // tracking policy of §IV-B applied inside the rollout (null gains: open loop): at step k the
    // control is pol_ubar[j] - pol_gains[j] . (x_k - pol_xbar[j]), j = pol_offset + k, plus the
    // open-loop control if `controls` is also given
    const double *pol_gains, *pol_xbar;
    const float *pol_ubar;
    int pol_offset;
    // disturbance pair count (0 or 2: the first two records are the pair) of the roots and of
    // the written-back states, indexed like root_n and out_n (null: none)
    const int *root_ndist;
    int *out_ndist;
    // binary32 path: per-block scratch of the pair sums (rev_stride float2 slots per block,
    // at least rollout_rev_slots(cap); null: the launcher allocates it around the launch)
    float2 *rev;
    long long rev_stride;
    // pacing of the co-resident blocks of a one-wave launch (null: off): per SM id below
    // pace_sms, a mask of the occupied slots and the step each slot's block has reached
    unsigned *pace_mask;
    int *pace_prog;             // pace_sms x kPaceSlots
    int pace_sms;
};
// Puts a disturbance pair in front of the n records of a state (one block): records move up by
// two, the pair takes slots 0 and 1, the count and the pair count are updated on the device.
cudaError_t launch_inject_pair(int precision, void *d_part, int *d_n, int cap, const double *pair,
                               cudaStream_t s);

size_t rollout_smem_bytes(int precision, int cap);
// The library's memory pool on the current device (null if it cannot be made) and a
// stream-ordered allocation from it; freed with cudaFreeAsync. Freed memory stays reserved in the
// pool for the library's next allocations; lib_pool_idle_bytes() is that reserved, unused part.
cudaMemPool_t lib_pool();
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);
size_t lib_pool_idle_bytes();
// float2 slots of pair-sum scratch one block of the binary32 path needs for capacity cap
// (0: none; the binary64 path needs none).
long long rollout_rev_slots(int precision, int cap);
// Scratch slot (float2 units) of a binary32 block with capacity cap: kind 0 = the first of the
// two slots of target `particle`'s forward sum; kind 1 = source `particle`'s reverse sum over row `row`.
long long rollout_scratch_slot(int cap, int kind, int row, int particle);
cudaError_t launch_rollout(int precision, const RolloutArgs &a, int grid, cudaStream_t s);
// Persistent launch over a.n_items rollouts with `nt` threads per block (128, 256 or 512; the
// binary64 path uses 128) and diagonal pair units of 32 dt targets (dt = 1, 2 or 4: every
// target's sum is formed in the same order whatever dt, so results do not change; dt other than
// 2 runs as 2 except for the Vatistas kernel); `grid` blocks claim rollouts in a.order through
// a.counter.
cudaError_t launch_uneven(int precision, const RolloutArgs &a, int grid, int nt, int dt, cudaStream_t s);
// Resident blocks per SM of the persistent kernel for this configuration (0 if it cannot run).
int uneven_blocks_per_sm(int precision, int kernel, int nt, int dt, size_t smem);
// The persistent launch with one rollout per cluster of `ctas` CTAs (2 or 4; binary32, Vatistas
// kernel only): `clusters` clusters claim rollouts; a.rev holds one scratch area per cluster.
// Results are the same bits as launch_uneven's.
cudaError_t launch_uneven_cluster(const RolloutArgs &a, int clusters, int nt, int dt, int ctas,
                                  cudaStream_t s);
// Clusters of `ctas` CTAs that can be resident at once for this configuration (0: it cannot run).
int uneven_max_clusters(int precision, int kernel, int nt, int dt, int ctas, size_t smem);
// Throughput probe of the binary32 pair loop (Vatistas kernel, core radius r_core): `grid`
// blocks of 128 threads each load the n records of d_src into shared memory and form every
// target's sum over all n sources `reps` times with t targets per lane (1, 2 or 4); block b
// writes its raw sums to d_out[b n ...].
cudaError_t launch_pair_probe(int t, int grid, int n, int reps, double r_core, const float4 *d_src,
                              float2 *d_out, cudaStream_t s);
// The pair phase of the binary32 rollout kernel itself (one evaluation per particle pair across
// rows, d_scratch holding grid x rollout_rev_slots(VPM_FP32, n) float2), `reps` times.
cudaError_t launch_pair_probe_sym(int grid, int n, int reps, double r_core, const float4 *d_src,
                                  float2 *d_out, float2 *d_scratch, cudaStream_t s);

}  // namespace vpm
