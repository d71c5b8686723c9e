// Free-field Biot-Savart velocities (Eq. 3 with the kernels of Eqs. 4-5) for large fields and
// their Heun time stepping, in two forms.
//
// Once per target (freefield_kernel, the allocation-free entry point's form): each thread holds
// two targets in registers; a block stages source tiles in shared memory with coalesced float4
// loads, every thread then reads each source by a broadcast shared-memory load. Plain binary32
// sums within a tile are added into Kahan-compensated totals across tiles.
//
// Once per pair (freefield_sym_kernel + freefield_combine_kernel, below): the form of
// vpm_freefield_velocity and vpm_freefield_heun.
#include "vpm_device.cuh"

namespace vpm {

constexpr int kFfThreads = 256;
constexpr int kFfTile = 512;   // sources staged per tile (8 KB)

// Epilogue modes of one velocity evaluation.
enum FfMode : int {
    kFfVelocity = 0,   // vel = V(src)
    kFfHeunStage1 = 1, // vel = V(src); mid = src + dt vel
    kFfHeunStage2 = 2  // out = out + dt/2 (vel + V(src)), src being the stage-1 positions
};

struct FfArgs {
    const float4 *src;   // sources and targets (x, z, Gamma, unused)
    int n;
    float rc4, inv_rc2;
    float dt;
    float2 *vel;         // velocity mode and stage 1: output; stage 2: v1 input
    float4 *mid;         // stage 1 output
    float4 *out;         // stage 2 output (in place over the base positions)
};

template <int KER, int MODE>
__global__ void __launch_bounds__(kFfThreads) freefield_kernel(const FfArgs a)
{
    __shared__ float4 tile[kFfTile];
    const int ia = blockIdx.x * (2 * kFfThreads) + threadIdx.x;
    const int ib = ia + kFfThreads;
    const int n = a.n;
    const float4 pa = a.src[ia < n ? ia : 0];
    const float4 pb = a.src[ib < n ? ib : 0];
    float sua = 0.f, cua = 0.f, swa = 0.f, cwa = 0.f;
    float sub = 0.f, cub = 0.f, swb = 0.f, cwb = 0.f;
    for (int j0 = 0; j0 < n; j0 += kFfTile) {
        const int cnt = min(kFfTile, n - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += kFfThreads) tile[t] = a.src[j0 + t];
        __syncthreads();
        float ua = 0.f, wa = 0.f, ub = 0.f, wb = 0.f;
#pragma unroll 8
        for (int j = 0; j < cnt; ++j) {
            const float4 s = tile[j];
            const float dxa = pa.x - s.x, dza = pa.y - s.y;
            const float dxb = pb.x - s.x, dzb = pb.y - s.y;
            const float ga = s.z * PairF32<KER>::q(fmaf(dxa, dxa, dza * dza), a.rc4, a.inv_rc2);
            const float gb = s.z * PairF32<KER>::q(fmaf(dxb, dxb, dzb * dzb), a.rc4, a.inv_rc2);
            ua = fmaf(-dza, ga, ua);
            wa = fmaf(dxa, ga, wa);
            ub = fmaf(-dzb, gb, ub);
            wb = fmaf(dxb, gb, wb);
        }
        kahan_add(sua, cua, ua);
        kahan_add(swa, cwa, wa);
        kahan_add(sub, cub, ub);
        kahan_add(swb, cwb, wb);
    }
    const float inv2pi = (float)kInv2Pi;
    const float va_u = (sua - cua) * inv2pi, va_w = (swa - cwa) * inv2pi;
    const float vb_u = (sub - cub) * inv2pi, vb_w = (swb - cwb) * inv2pi;
    if (MODE == kFfVelocity) {
        if (ia < n) a.vel[ia] = make_float2(va_u, va_w);
        if (ib < n) a.vel[ib] = make_float2(vb_u, vb_w);
    } else if (MODE == kFfHeunStage1) {
        if (ia < n) {
            a.vel[ia] = make_float2(va_u, va_w);
            a.mid[ia] = make_float4(fmaf(a.dt, va_u, pa.x), fmaf(a.dt, va_w, pa.y), pa.z, 0.f);
        }
        if (ib < n) {
            a.vel[ib] = make_float2(vb_u, vb_w);
            a.mid[ib] = make_float4(fmaf(a.dt, vb_u, pb.x), fmaf(a.dt, vb_w, pb.y), pb.z, 0.f);
        }
    } else {
        const float h = 0.5f * a.dt;
        if (ia < n) {
            const float2 v1 = a.vel[ia];
            float4 q = a.out[ia];
            q.x = fmaf(h, v1.x + va_u, q.x);
            q.y = fmaf(h, v1.y + va_w, q.y);
            a.out[ia] = q;
        }
        if (ib < n) {
            const float2 v1 = a.vel[ib];
            float4 q = a.out[ib];
            q.x = fmaf(h, v1.x + vb_u, q.x);
            q.y = fmaf(h, v1.y + vb_w, q.y);
            a.out[ib] = q;
        }
    }
}

template <int MODE>
static cudaError_t launch_mode(int kernel, const FfArgs &a, cudaStream_t s)
{
    const int grid = (a.n + 2 * kFfThreads - 1) / (2 * kFfThreads);
    if (grid == 0) return cudaSuccess;
    if (kernel == VPM_KERNEL_GAUSSIAN)
        freefield_kernel<VPM_KERNEL_GAUSSIAN, MODE><<<grid, kFfThreads, 0, s>>>(a);
    else if (kernel == VPM_KERNEL_SINGULAR)
        freefield_kernel<VPM_KERNEL_SINGULAR, MODE><<<grid, kFfThreads, 0, s>>>(a);
    else
        freefield_kernel<VPM_KERNEL_VATISTAS, MODE><<<grid, kFfThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Heun steps with caller-provided scratch: mid[n] float4 and v1[n] float2.
cudaError_t launch_freefield_heun(float *p, int n, int kernel, double r_core, double dt,
                                  int steps, float *scratch_mid, float *scratch_v1,
                                  cudaStream_t s)
{
    FfArgs a{};
    a.n = n;
    a.rc4 = (float)(r_core * r_core * r_core * r_core);
    a.inv_rc2 = r_core > 0 ? (float)(1.0 / (r_core * r_core)) : 0.f;
    a.dt = (float)dt;
    a.vel = reinterpret_cast<float2 *>(scratch_v1);
    a.mid = reinterpret_cast<float4 *>(scratch_mid);
    a.out = reinterpret_cast<float4 *>(p);
    for (int k = 0; k < steps; ++k) {
        a.src = reinterpret_cast<const float4 *>(p);
        cudaError_t e = launch_mode<kFfHeunStage1>(kernel, a, s);
        if (e != cudaSuccess) return e;
        a.src = a.mid;
        e = launch_mode<kFfHeunStage2>(kernel, a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------ one evaluation per pair
//
// The pair factor depends on the distance only and the displacement changes sign with the
// roles of the two particles, so one evaluation of a pair serves both particles' sums.
//
// The n particles form rows of kFsRow = 1024 (row I: particles 1024 I ..), one per CTA of 8
// warps, each warp holding 128 of them (4 per lane). Sources are staged in shared memory in
// tiles of kFsTile = 512 and visited in blocks of 32, two blocks per rotation: in round r lane
// l takes source (l + r) mod 32 of each block, adds the forward terms to its 4 targets and the
// reverse terms to the sources' running sums, which then move one lane down. After a tile the
// 8 warps' reverse sums of each source are added in warp order in shared memory.
//   * off-diagonal units (row I, segment s): the row against kFsSeg tiles of later particles;
//     the reverse sums go to the slot of (row I, source), the targets' compensated sums over
//     the segment to the slot of (row I, segment, target);
//   * diagonal unit (row I): the row against itself. Warp w takes the 32-blocks of warps
//     w' > w by rotation and its own 4 blocks once per target (both orders), and leaves the
//     blocks of warps w' < w to them; the reverse sums go to the slot of the source.
// A second kernel adds, per particle, its diagonal sums, its row's segment sums and the
// reverse sums of every earlier row, in that order (Kahan), and applies the step's epilogue.
// Every partial sum is formed in a fixed order, so results do not depend on scheduling.
constexpr int kFsWarps = 8, kFsThreads = 32 * kFsWarps;
constexpr int kFsRow = 128 * kFsWarps;      // targets of a row (4 per lane)
constexpr int kFsTile = 512;                // sources per staged tile (16 blocks of 32)
constexpr int kFsSeg = 32;                  // tiles per off-diagonal unit (16384 sources)
#ifndef VPM_FS_MIN_BLOCKS
#define VPM_FS_MIN_BLOCKS 4
#endif

struct FsGeom {
    int n, rows, ntiles, max_seg;           // rows = ceil(n / kFsRow), ntiles = ceil(n / kFsTile)
    long long f_seg, r_slot, total;         // float2 offsets: [diag fwd n][diag rev n][seg][rev]
};

__host__ __device__ inline FsGeom fs_geom(int n)
{
    FsGeom g;
    g.n = n;
    g.rows = (n + kFsRow - 1) / kFsRow;
    g.ntiles = (n + kFsTile - 1) / kFsTile;
    // row 0 has the most off-diagonal tiles: ntiles - 2 (the row spans two tiles)
    const int t0 = g.ntiles - kFsRow / kFsTile;
    g.max_seg = t0 > 0 ? (t0 + kFsSeg - 1) / kFsSeg : 0;
    g.f_seg = 2LL * n;
    g.r_slot = g.f_seg + (long long)g.rows * g.max_seg * kFsRow;
    // reverse slots of row I: sources kFsRow (I + 1) .. ntiles kFsTile - 1
    const long long span = (long long)g.ntiles * kFsTile;
    const long long R = g.rows > 1 ? g.rows - 1 : 0;       // rows with later particles
    g.total = g.r_slot + R * span - (long long)kFsRow * R * (R + 1) / 2;
    return g;
}

__host__ __device__ inline long long fs_rev_base(const FsGeom &g, int I)
{
    const long long span = (long long)g.ntiles * kFsTile;
    return g.r_slot + (long long)I * span - (long long)kFsRow * I * (I + 1) / 2 - (long long)kFsRow * (I + 1);
}

// Stages sources t0 .. t0 + kFsTile - 1 (past n: the last particle's position, zero strength).
__device__ __forceinline__ void fs_stage(float4 *tile, const float4 *src, int n, int t0)
{
    const float4 last = src[n - 1];
    for (int t = threadIdx.x; t < kFsTile; t += kFsThreads) {
        const int j = t0 + t;
        float4 v = j < n ? src[j] : last;
        if (j >= n) v.z = 0.f;
        tile[t] = v;
    }
}

// One block (b0 .. b0+31 of the tile) by rotation; returns lane l's reverse sum of source b0+l.
template <int KER>
__device__ __forceinline__ float2 fs_rotate_one(const float4 *tile, int b0, float rc4, float irc2,
                                                const float (&tx)[4], const float (&tz)[4],
                                                const float (&tg)[4], float (&fu)[4], float (&fw)[4])
{
    const int lane = threadIdx.x & 31;
    float ru = 0.f, rw = 0.f;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const float4 s = tile[b0 + ((lane + r) & 31)];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s.x, dz = tz[k] - s.y;
            const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
            const float gs = s.z * q, gt = tg[k] * q;
            fu[k] = fmaf(-dz, gs, fu[k]);
            fw[k] = fmaf(dx, gs, fw[k]);
            ru = fmaf(dz, gt, ru);
            rw = fmaf(-dx, gt, rw);
        }
        ru = __shfl_sync(0xffffffffu, ru, (lane + 1) & 31);
        rw = __shfl_sync(0xffffffffu, rw, (lane + 1) & 31);
    }
    return make_float2(ru, rw);
}

// Two blocks (b0 .. b0+63 of the tile) by rotation, one source of each per round.
template <int KER>
__device__ __forceinline__ void fs_rotate_two(const float4 *tile, int b0, float rc4, float irc2,
                                              const float (&tx)[4], const float (&tz)[4],
                                              const float (&tg)[4], float (&fu)[4], float (&fw)[4],
                                              float2 &r1, float2 &r2)
{
    const int lane = threadIdx.x & 31;
    float ru1 = 0.f, rw1 = 0.f, ru2 = 0.f, rw2 = 0.f;
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
        const int j = b0 + ((lane + r) & 31);
        const float4 s1 = tile[j], s2 = tile[j + 32];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s1.x, dz = tz[k] - s1.y;
            const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
            const float gs = s1.z * q, gt = tg[k] * q;
            fu[k] = fmaf(-dz, gs, fu[k]);
            fw[k] = fmaf(dx, gs, fw[k]);
            ru1 = fmaf(dz, gt, ru1);
            rw1 = fmaf(-dx, gt, rw1);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s2.x, dz = tz[k] - s2.y;
            const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
            const float gs = s2.z * q, gt = tg[k] * q;
            fu[k] = fmaf(-dz, gs, fu[k]);
            fw[k] = fmaf(dx, gs, fw[k]);
            ru2 = fmaf(dz, gt, ru2);
            rw2 = fmaf(-dx, gt, rw2);
        }
        ru1 = __shfl_sync(0xffffffffu, ru1, (lane + 1) & 31);
        rw1 = __shfl_sync(0xffffffffu, rw1, (lane + 1) & 31);
        ru2 = __shfl_sync(0xffffffffu, ru2, (lane + 1) & 31);
        rw2 = __shfl_sync(0xffffffffu, rw2, (lane + 1) & 31);
    }
    r1 = make_float2(ru1, rw1);
    r2 = make_float2(ru2, rw2);
}

// One block once per target (its sources' reverse terms are not formed).
template <int KER>
__device__ __forceinline__ void fs_direct_block(const float4 *tile, int b0, float rc4, float irc2,
                                                const float (&tx)[4], const float (&tz)[4],
                                                float (&fu)[4], float (&fw)[4])
{
#pragma unroll 4
    for (int j = b0; j < b0 + 32; ++j) {
        const float4 s = tile[j];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s.x, dz = tz[k] - s.y;
            const float g = s.z * PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
            fu[k] = fmaf(-dz, g, fu[k]);
            fw[k] = fmaf(dx, g, fw[k]);
        }
    }
}

__device__ __forceinline__ void fs_fold(float (&su)[4], float (&cu)[4], float (&sw)[4],
                                        float (&cw)[4], float (&fu)[4], float (&fw)[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        kahan_add(su[k], cu[k], fu[k]);
        kahan_add(sw[k], cw[k], fw[k]);
        fu[k] = fw[k] = 0.f;
    }
}

// grid (1 + max_seg, rows): x = 0 the diagonal unit of row y, x = s + 1 its segment s.
template <int KER>
__global__ void __launch_bounds__(kFsThreads, VPM_FS_MIN_BLOCKS)
freefield_sym_kernel(const float4 *src, int n, float rc4, float irc2, float2 *scr)
{
    __shared__ float4 tile[kFsTile];
    __shared__ float2 stage[kFsWarps][kFsTile];
    const FsGeom g = fs_geom(n);
    const int I = blockIdx.y, unit = blockIdx.x;
    const int tr0 = I * (kFsRow / kFsTile);                 // the row's first tile
    int t_begin, t_end;
    if (unit == 0) {
        t_begin = tr0;
        t_end = min(tr0 + kFsRow / kFsTile, g.ntiles);
    } else {
        t_begin = tr0 + kFsRow / kFsTile + (unit - 1) * kFsSeg;
        t_end = min(t_begin + kFsSeg, g.ntiles);
        if (t_begin >= t_end) return;                      // the row has fewer segments
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float4 last = src[n - 1];
    float tx[4], tz[4], tg[4], su[4], cu[4], sw[4], cw[4], fu[4], fw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = I * kFsRow + 128 * warp + 32 * k + lane;
        float4 q = i < n ? src[i] : last;
        tx[k] = q.x;
        tz[k] = q.y;
        tg[k] = i < n ? q.z : 0.f;
        su[k] = cu[k] = sw[k] = cw[k] = fu[k] = fw[k] = 0.f;
    }
    for (int t = t_begin; t < t_end; ++t) {
        __syncthreads();                                   // the previous tile is consumed
        fs_stage(tile, src, n, t * kFsTile);
        __syncthreads();
        if (unit == 0) {
            // block gb of the row (0 .. 31) belongs to warp gb / 4
            for (int b = 0; b < kFsTile / 32; ++b) {
                const int gb = (t - tr0) * (kFsTile / 32) + b, owner = gb >> 2;
                float2 r = make_float2(0.f, 0.f);
                if (owner > warp)
                    r = fs_rotate_one<KER>(tile, 32 * b, rc4, irc2, tx, tz, tg, fu, fw);
                else if (owner == warp)
                    fs_direct_block<KER>(tile, 32 * b, rc4, irc2, tx, tz, fu, fw);
                stage[warp][32 * b + lane] = r;
                if (b & 1) fs_fold(su, cu, sw, cw, fu, fw);
            }
        } else {
            for (int b = 0; b < kFsTile / 32; b += 2) {
                float2 r1, r2;
                fs_rotate_two<KER>(tile, 32 * b, rc4, irc2, tx, tz, tg, fu, fw, r1, r2);
                stage[warp][32 * b + lane] = r1;
                stage[warp][32 * b + 32 + lane] = r2;
                fs_fold(su, cu, sw, cw, fu, fw);
            }
        }
        __syncthreads();
        // the warps' reverse sums of every source of the tile, added in warp order
        for (int q = threadIdx.x; q < kFsTile; q += kFsThreads) {
            const int j = t * kFsTile + q;
            if (j >= n) continue;
            float ru = 0.f, rw = 0.f;
#pragma unroll
            for (int w = 0; w < kFsWarps; ++w) {
                ru += stage[w][q].x;
                rw += stage[w][q].y;
            }
            if (unit == 0) scr[(long long)n + j] = make_float2(ru, rw);
            else scr[fs_rev_base(g, I) + j] = make_float2(ru, rw);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int li = 128 * warp + 32 * k + lane, i = I * kFsRow + li;
        if (i >= n) continue;
        const float2 f = make_float2(su[k] - cu[k], sw[k] - cw[k]);
        if (unit == 0) scr[i] = f;
        else scr[g.f_seg + ((long long)I * g.max_seg + (unit - 1)) * kFsRow + li] = f;
    }
}

// Per particle: every partial sum in a fixed order, then the evaluation's epilogue.
template <int MODE>
__global__ void __launch_bounds__(256) freefield_combine_kernel(const FfArgs a, const float2 *scr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    if (j >= n) return;
    const FsGeom g = fs_geom(n);
    const int T = j / kFsRow, li = j - T * kFsRow;
    float2 v = scr[j];
    float cu = 0.f, cw = 0.f;
    {
        const float2 d = scr[(long long)n + j];
        kahan_add(v.x, cu, d.x);
        kahan_add(v.y, cw, d.y);
    }
    // the row's segments: those that exist (tiles after the row's own two)
    const int t_after = g.ntiles - (T + 1) * (kFsRow / kFsTile);
    const int segs = t_after > 0 ? (t_after + kFsSeg - 1) / kFsSeg : 0;
    for (int s = 0; s < segs; ++s) {
        const float2 f = scr[g.f_seg + ((long long)T * g.max_seg + s) * kFsRow + li];
        kahan_add(v.x, cu, f.x);
        kahan_add(v.y, cw, f.y);
    }
    int I = 0;
    for (; I + 4 <= T; I += 4) {                           // four loads in flight
        float2 r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = scr[fs_rev_base(g, I + q) + j];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            kahan_add(v.x, cu, r[q].x);
            kahan_add(v.y, cw, r[q].y);
        }
    }
    for (; I < T; ++I) {
        const float2 r = scr[fs_rev_base(g, I) + j];
        kahan_add(v.x, cu, r.x);
        kahan_add(v.y, cw, r.y);
    }
    const float inv2pi = (float)kInv2Pi;
    const float vu = (v.x - cu) * inv2pi, vw = (v.y - cw) * inv2pi;
    if (MODE == kFfVelocity) {
        a.vel[j] = make_float2(vu, vw);
    } else if (MODE == kFfHeunStage1) {
        const float4 p = a.src[j];
        a.vel[j] = make_float2(vu, vw);
        a.mid[j] = make_float4(fmaf(a.dt, vu, p.x), fmaf(a.dt, vw, p.y), p.z, 0.f);
    } else {
        const float h = 0.5f * a.dt;
        const float2 v1 = a.vel[j];
        float4 q = a.out[j];
        q.x = fmaf(h, v1.x + vu, q.x);
        q.y = fmaf(h, v1.y + vw, q.y);
        a.out[j] = q;
    }
}

size_t freefield_sym_scratch_bytes(int n)
{
    return n > 0 ? sizeof(float2) * (size_t)fs_geom(n).total : 0;
}

template <int MODE>
static cudaError_t sym_eval(int kernel, const FfArgs &a, float2 *scr, cudaStream_t s)
{
    const FsGeom g = fs_geom(a.n);
    if (a.n == 0) return cudaSuccess;
    const dim3 grid(1 + g.max_seg, g.rows);
    if (kernel == VPM_KERNEL_GAUSSIAN)
        freefield_sym_kernel<VPM_KERNEL_GAUSSIAN><<<grid, kFsThreads, 0, s>>>(a.src, a.n, a.rc4, a.inv_rc2, scr);
    else if (kernel == VPM_KERNEL_SINGULAR)
        freefield_sym_kernel<VPM_KERNEL_SINGULAR><<<grid, kFsThreads, 0, s>>>(a.src, a.n, a.rc4, a.inv_rc2, scr);
    else
        freefield_sym_kernel<VPM_KERNEL_VATISTAS><<<grid, kFsThreads, 0, s>>>(a.src, a.n, a.rc4, a.inv_rc2, scr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    freefield_combine_kernel<MODE><<<(a.n + 255) / 256, 256, 0, s>>>(a, scr);
    return cudaGetLastError();
}

// Velocities with one evaluation per pair; scratch: freefield_sym_scratch_bytes(n).
cudaError_t launch_freefield_sym_velocity(const float *p, int n, int kernel, double r_core,
                                          float *vel, void *scratch, cudaStream_t s)
{
    FfArgs a{};
    a.src = reinterpret_cast<const float4 *>(p);
    a.n = n;
    a.rc4 = (float)(r_core * r_core * r_core * r_core);
    a.inv_rc2 = r_core > 0 ? (float)(1.0 / (r_core * r_core)) : 0.f;
    a.vel = reinterpret_cast<float2 *>(vel);
    return sym_eval<kFfVelocity>(kernel, a, static_cast<float2 *>(scratch), s);
}

// Heun steps with one evaluation per pair; scratch_mid[n] float4, scratch_v1[n] float2 and
// the pair-sum scratch of freefield_sym_scratch_bytes(n).
cudaError_t launch_freefield_sym_heun(float *p, int n, int kernel, double r_core, double dt,
                                      int steps, float *scratch_mid, float *scratch_v1,
                                      void *scratch, cudaStream_t s)
{
    FfArgs a{};
    a.n = n;
    a.rc4 = (float)(r_core * r_core * r_core * r_core);
    a.inv_rc2 = r_core > 0 ? (float)(1.0 / (r_core * r_core)) : 0.f;
    a.dt = (float)dt;
    a.vel = reinterpret_cast<float2 *>(scratch_v1);
    a.mid = reinterpret_cast<float4 *>(scratch_mid);
    a.out = reinterpret_cast<float4 *>(p);
    float2 *scr = static_cast<float2 *>(scratch);
    for (int k = 0; k < steps; ++k) {
        a.src = reinterpret_cast<const float4 *>(p);
        cudaError_t e = sym_eval<kFfHeunStage1>(kernel, a, scr, s);
        if (e != cudaSuccess) return e;
        a.src = a.mid;
        e = sym_eval<kFfHeunStage2>(kernel, a, scr, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace vpm
