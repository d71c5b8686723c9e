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
#include <string.h>

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
    int kernel;          // vpm_kernel (the one-evaluation-per-pair form's scale)
    float r_core;
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
//     the targets' sums over the segment are Kahan-compensated across the tiles;
//   * diagonal unit (row I): the row against itself. Warp w takes the 32-blocks of warps
//     w' > w by rotation and its own 4 blocks once per target (both orders), and leaves the
//     blocks of warps w' < w to them.
// Every partial sum (a tile's reverse sums of a source, a unit's forward sums of a target) is
// added into its particle's exact accumulator: a fixed-point integer per velocity component,
// held as three signed 64-bit digit words of radix 2^42, 48 bytes per particle. Integer
// addition is exact and associative, so each particle's total is the exact sum of its binary32
// partial sums whatever order the CTAs run in, and the scratch grows like n, not like n^2. A second kernel turns each accumulator into
// the velocity, applies the step's epilogue and clears the accumulator for the next evaluation.
constexpr int kFsWarps = 8, kFsThreads = 32 * kFsWarps;
constexpr int kFsRow = 128 * kFsWarps;      // targets of a row (4 per lane)
constexpr int kFsTile = 512;                // sources per staged tile (16 blocks of 32)
constexpr int kFsSeg = 32;                  // tiles per off-diagonal unit (16384 sources)
#ifndef VPM_FS_MIN_BLOCKS
#define VPM_FS_MIN_BLOCKS 4
#endif

struct FsGeom {
    int n, rows, ntiles, max_seg;           // rows = ceil(n / kFsRow), ntiles = ceil(n / kFsTile)
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
    return g;
}

// ------------------------------------------------------------------ exact accumulation
//
// A particle's accumulator holds its velocity sums (u, w) in units of 2^-e as integers, each
// kept as kFsDigits signed 64-bit words d_0, d_1, d_2 of weight 2^0, 2^42, 2^84 (acc[6 j + 0..2]
// for u, [6 j + 3..5] for w): the value is d_0 + d_1 2^42 + d_2 2^84 as a 128-bit integer. A
// partial sum's integer has 24 significant bits, so it adds a digit below 2^42 to at most two
// words, with a plain 64-bit reduction each (no carry between words, no atomic with return).
// A word stays exact while it receives fewer than 2^21 additions: a particle receives one per
// row of 1024 particles before its own plus one per unit of its own row (at most n / 1024 +
// n / 16384 + 3 for n particles), below 2^21 for n <= kFsMaxN = 2^30. The exponent e is fixed for a call by a bound B on every partial sum and on every total: no term
// of the sums exceeds max|Gamma| kappa, with kappa = 1 / r_core for the regularised kernels
// (|r q(r)| peaks at 1 / (sqrt(2) r_core) for Eq. 5 and at 0.64 / r_core for the Gaussian core)
// and 2^40 for the singular kernel (distances down to 2^-40), so |sum| <= B = n max|Gamma| kappa.
// With B < 2^eb, e = 125 - eb keeps every value below 2^126 and the resolution at B 2^-125.
constexpr int kFsDigitBits = 42, kFsDigits = 3, kFsWords = 2 * kFsDigits;
constexpr int kFsMaxN = 1 << 30;

struct FsScale {
    int gmax_bits;                          // max |Gamma| of the call (binary32 bits, >= 0)
    int nonfinite;                          // set when a partial sum is NaN or infinite
    int pad[14];
};

__host__ __device__ inline int fs_exponent(float gmax, int n, int kernel, float r_core)
{
    if (!(gmax > 0.f) || n <= 0) return 0;
    const double kappa = kernel == VPM_KERNEL_SINGULAR ? 1099511627776.0 : 1.0 / (double)r_core;
    const double B = (double)n * (double)gmax * kappa;
    if (!(B < 1e300)) return 0;
    int eb = 0;
    frexp(B, &eb);                          // B < 2^eb
    return 125 - eb;
}

// v 2^e as a 128-bit two's-complement integer (lo, hi), rounded to nearest (half away from
// zero) below the unit; bad is set for NaN and infinities. Zero and subnormal v give 0.
__host__ __device__ inline void fs_to_fixed(float v, int e, unsigned long long &lo,
                                            unsigned long long &hi, bool &bad)
{
    unsigned b;
    memcpy(&b, &v, sizeof b);
    const int ex = (int)((b >> 23) & 0xffu);
    lo = hi = 0ull;
    if (ex == 0xff) { bad = true; return; }
    if (ex == 0) return;
    const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | 0x800000u);   // v = m 2^(ex-150)
    const int sh = ex - 150 + e;
    if (sh >= 64) {
        hi = m << (sh - 64);
    } else if (sh > 40) {
        lo = m << sh;
        hi = m >> (64 - sh);
    } else if (sh >= 0) {
        lo = m << sh;
    } else if (sh > -25) {
        lo = (m + (1ull << (-sh - 1))) >> (-sh);
    }
    if (b >> 31) {                          // negate: two's complement over 128 bits
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
}

// The digits of v 2^e (v's integer from fs_to_fixed): the value's 128 bits cut at bits 42 and
// 84. Each digit is added to its word as a signed 64-bit integer (two's complement).
__host__ __device__ inline void fs_to_digits(float v, int e, unsigned long long (&d)[kFsDigits], bool &bad)
{
    unsigned long long lo, hi;
    fs_to_fixed(fabsf(v), e, lo, hi, bad);
    const unsigned long long mask = (1ull << kFsDigitBits) - 1ull;
    d[0] = lo & mask;
    d[1] = ((lo >> kFsDigitBits) | (hi << (64 - kFsDigitBits))) & mask;
    d[2] = hi >> (2 * kFsDigitBits - 64);
    if (signbit(v)) {
        for (int k = 0; k < kFsDigits; ++k) d[k] = 0ull - d[k];
    }
}

// The digit words w[0..2] as one 128-bit two's-complement integer (lo, hi).
__host__ __device__ inline void fs_from_digits(const unsigned long long (&w)[kFsDigits],
                                               unsigned long long &lo, unsigned long long &hi)
{
    lo = hi = 0ull;
    for (int k = 0; k < kFsDigits; ++k) {
        const int sh = kFsDigitBits * k;
        const unsigned long long x = w[k], ext = (long long)x < 0 ? ~0ull : 0ull;   // sign extension
        const unsigned long long xl = sh >= 64 ? 0ull : (sh ? x << sh : x);
        const unsigned long long xh = sh >= 64 ? x << (sh - 64) : (sh ? (x >> (64 - sh)) | (ext << sh) : ext);
        const unsigned long long old = lo;
        lo += xl;
        hi += xh + (lo < old ? 1ull : 0ull);
    }
}

// The accumulator (lo, hi) as a double (one rounding), in units of 1.
__host__ __device__ inline double fs_from_fixed(unsigned long long lo, unsigned long long hi, int e)
{
    const bool neg = (long long)hi < 0;
    if (neg) {
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    const double d = ldexp((double)hi, 64) + (double)lo;
    return ldexp(neg ? -d : d, -e);
}

// Adds v (units of 1) to the digit words at a: concurrent additions in any order leave the
// exact sum (each word's additions commute; nothing carries between words until the combine).
__device__ __forceinline__ void fs_acc_add(unsigned long long *a, float v, int e, int *nonfinite)
{
    unsigned long long d[kFsDigits];
    bool bad = false;
    fs_to_digits(v, e, d, bad);
    if (bad) {
        atomicOr(nonfinite, 1);
        return;
    }
#pragma unroll
    for (int k = 0; k < kFsDigits; ++k)
        if (d[k]) atomicAdd(a + k, d[k]);
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
freefield_sym_kernel(const float4 *src, int n, float rc4, float irc2, unsigned long long *acc,
                     FsScale *scale, int kernel, float r_core)
{
    __shared__ float4 tile[kFsTile];
    __shared__ float2 stage[kFsWarps][kFsTile];
    __shared__ int s_e;
    const FsGeom g = fs_geom(n);
    if (threadIdx.x == 0) s_e = fs_exponent(__int_as_float(scale->gmax_bits), n, kernel, r_core);
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
            fs_acc_add(acc + kFsWords * (size_t)j, ru, s_e, &scale->nonfinite);
            fs_acc_add(acc + kFsWords * (size_t)j + kFsDigits, rw, s_e, &scale->nonfinite);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = I * kFsRow + 128 * warp + 32 * k + lane;
        if (i >= n) continue;
        fs_acc_add(acc + kFsWords * (size_t)i, su[k] - cu[k], s_e, &scale->nonfinite);
        fs_acc_add(acc + kFsWords * (size_t)i + kFsDigits, sw[k] - cw[k], s_e, &scale->nonfinite);
    }
}

// Per particle: the exact sums as velocities, the evaluation's epilogue, and the accumulator
// cleared for the next evaluation of the call.
template <int MODE>
__global__ void __launch_bounds__(256) freefield_combine_kernel(const FfArgs a, unsigned long long *acc,
                                                                 const FsScale *scale)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = a.n;
    if (j >= n) return;
    const int e = fs_exponent(__int_as_float(scale->gmax_bits), n, a.kernel, a.r_core);
    unsigned long long *q = acc + kFsWords * (size_t)j;
    unsigned long long du[kFsDigits], dw[kFsDigits], ul, uh, wl, wh;
#pragma unroll
    for (int k = 0; k < kFsDigits; ++k) {
        du[k] = q[k];
        dw[k] = q[kFsDigits + k];
        q[k] = q[kFsDigits + k] = 0ull;
    }
    fs_from_digits(du, ul, uh);
    fs_from_digits(dw, wl, wh);
    const double su = fs_from_fixed(ul, uh, e), sw = fs_from_fixed(wl, wh, e);
    float vu = (float)(su * kInv2Pi), vw = (float)(sw * kInv2Pi);
    if (scale->nonfinite) vu = vw = __int_as_float(0x7fc00000);
    if (MODE == kFfVelocity) {
        a.vel[j] = make_float2(vu, vw);
    } else if (MODE == kFfHeunStage1) {
        const float4 p = a.src[j];
        a.vel[j] = make_float2(vu, vw);
        a.mid[j] = make_float4(fmaf(a.dt, vu, p.x), fmaf(a.dt, vw, p.y), p.z, 0.f);
    } else {
        const float h = 0.5f * a.dt;
        const float2 v1 = a.vel[j];
        float4 p = a.out[j];
        p.x = fmaf(h, v1.x + vu, p.x);
        p.y = fmaf(h, v1.y + vw, p.y);
        a.out[j] = p;
    }
}

// max |Gamma| of the field (binary32 bits of non-negative floats order like the integers).
__global__ void __launch_bounds__(256) freefield_gmax_kernel(const float4 *src, int n, FsScale *scale)
{
    int m = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        m = max(m, __float_as_int(fabsf(src[j].z)));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&scale->gmax_bits, m);
}

// Scratch of one call: the accumulators (48 bytes per particle), then the call's scale.
constexpr size_t kFsAccBytes = sizeof(unsigned long long) * kFsWords;
size_t freefield_sym_scratch_bytes(int n)
{
    return n > 0 ? kFsAccBytes * (size_t)n + sizeof(FsScale) : 0;
}

int freefield_sym_max_n() { return kFsMaxN; }

// Zeroes the call's scratch and finds max |Gamma| (the strengths do not change during a call).
static cudaError_t sym_begin(const float4 *src, int n, void *scratch, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(scratch, 0, freefield_sym_scratch_bytes(n), s);
    if (e != cudaSuccess) return e;
    FsScale *scale = reinterpret_cast<FsScale *>(static_cast<unsigned char *>(scratch) + kFsAccBytes * (size_t)n);
    const int grid = min((n + 255) / 256, 1184);
    freefield_gmax_kernel<<<grid, 256, 0, s>>>(src, n, scale);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t sym_eval(int kernel, const FfArgs &a, void *scratch, cudaStream_t s)
{
    const FsGeom g = fs_geom(a.n);
    if (a.n == 0) return cudaSuccess;
    unsigned long long *acc = static_cast<unsigned long long *>(scratch);
    FsScale *scale = reinterpret_cast<FsScale *>(static_cast<unsigned char *>(scratch) + kFsAccBytes * (size_t)a.n);
    const dim3 grid(1 + g.max_seg, g.rows);
    if (kernel == VPM_KERNEL_GAUSSIAN)
        freefield_sym_kernel<VPM_KERNEL_GAUSSIAN><<<grid, kFsThreads, 0, s>>>(a.src, a.n, a.rc4, a.inv_rc2, acc, scale, kernel, a.r_core);
    else if (kernel == VPM_KERNEL_SINGULAR)
        freefield_sym_kernel<VPM_KERNEL_SINGULAR><<<grid, kFsThreads, 0, s>>>(a.src, a.n, a.rc4, a.inv_rc2, acc, scale, kernel, a.r_core);
    else
        freefield_sym_kernel<VPM_KERNEL_VATISTAS><<<grid, kFsThreads, 0, s>>>(a.src, a.n, a.rc4, a.inv_rc2, acc, scale, kernel, a.r_core);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    freefield_combine_kernel<MODE><<<(a.n + 255) / 256, 256, 0, s>>>(a, acc, scale);
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
    a.kernel = kernel;
    a.r_core = (float)r_core;
    a.vel = reinterpret_cast<float2 *>(vel);
    if (n == 0) return cudaSuccess;
    cudaError_t e = sym_begin(a.src, n, scratch, s);
    if (e != cudaSuccess) return e;
    return sym_eval<kFfVelocity>(kernel, a, scratch, s);
}

// Heun steps with one evaluation per pair; scratch_mid[n] float4, scratch_v1[n] float2 and
// the accumulators of freefield_sym_scratch_bytes(n).
cudaError_t launch_freefield_sym_heun(float *p, int n, int kernel, double r_core, double dt,
                                      int steps, float *scratch_mid, float *scratch_v1,
                                      void *scratch, cudaStream_t s)
{
    FfArgs a{};
    a.n = n;
    a.rc4 = (float)(r_core * r_core * r_core * r_core);
    a.inv_rc2 = r_core > 0 ? (float)(1.0 / (r_core * r_core)) : 0.f;
    a.kernel = kernel;
    a.r_core = (float)r_core;
    a.dt = (float)dt;
    a.vel = reinterpret_cast<float2 *>(scratch_v1);
    a.mid = reinterpret_cast<float4 *>(scratch_mid);
    a.out = reinterpret_cast<float4 *>(p);
    if (n == 0 || steps == 0) return cudaSuccess;
    cudaError_t e = sym_begin(reinterpret_cast<const float4 *>(p), n, scratch, s);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < steps; ++k) {
        a.src = reinterpret_cast<const float4 *>(p);
        e = sym_eval<kFfHeunStage1>(kernel, a, scratch, s);
        if (e != cudaSuccess) return e;
        a.src = a.mid;
        e = sym_eval<kFfHeunStage2>(kernel, a, scratch, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace vpm

// Host-side check of the exact accumulation (no device needed): the values h_v[count] converted
// with exponent e into the kernels' digits, added word by word in the given order as the kernels'
// reductions do, and the words combined into the 128-bit total, returned as a double.
extern "C" vpm_status vpm_fixed_sum(const float *h_v, int count, int e, double *h_sum, int *h_bad)
{
    if ((!h_v && count > 0) || count < 0 || !h_sum || !h_bad) return VPM_ERR_INVALID;
    unsigned long long w[vpm::kFsDigits] = {0ull, 0ull, 0ull};
    int bad = 0;
    for (int i = 0; i < count; ++i) {
        unsigned long long d[vpm::kFsDigits];
        bool b = false;
        vpm::fs_to_digits(h_v[i], e, d, b);
        if (b) { bad = 1; continue; }
        for (int k = 0; k < vpm::kFsDigits; ++k) w[k] += d[k];
    }
    unsigned long long lo, hi;
    vpm::fs_from_digits(w, lo, hi);
    *h_sum = vpm::fs_from_fixed(lo, hi, e);
    *h_bad = bad;
    return VPM_OK;
}

// The exponent the free-field kernels use for n particles of largest |Gamma| gmax.
extern "C" vpm_status vpm_fixed_exponent(float gmax, int n, int kernel, double r_core, int *h_e)
{
    if (!h_e || n < 0) return VPM_ERR_INVALID;
    *h_e = vpm::fs_exponent(gmax, n, kernel, (float)r_core);
    return VPM_OK;
}
