// Persistent rollout kernel: one block (128 threads on the MPPI batch; 256 or 512 for larger
// fields) advances one rollout of the coupled glider + VPM model (§III-A, §III-B) for the whole
// horizon with the field resident in shared memory, then writes the terminal cost (Eq. 24). The same step code serves vpm_step (one
// block, one step, state written back) and the one-rollout-per-launch comparison form.
//
// One step, in the order of §III-A: plate geometry from the glider state; relative velocity of
// Eq. 12 at the collocation and bound points from the wake before shedding; the surface
// circulation Gamma_S = K^-1 b of Eq. 11 with the body-frame inverse (K is constant in the
// body frame, so its inverse is formed once on the host); unsteady Bernoulli loads (Eqs.
// 13-15); the glider's explicit Euler update (Eqs. 18-22); LEV/TEV appended to the wake;
// convection velocities of Eq. 16 for every wake particle; explicit Euler advection and the
// decay of Eq. 17; merging of the two oldest particles while N > N_w,max.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdlib>
#include <mutex>

#include "vpm_rollout.cuh"

namespace vpm {

// Device-side bounds checks (build with -DVPM_DEBUG_BOUNDS=1): a record written past the
// block's capacity is skipped and the rollout's status gets the capacity flag (reported as
// VPM_ERR_CAPACITY); nothing traps. Off by default: the host's count bounds make them redundant.
#ifndef VPM_DEBUG_BOUNDS
#define VPM_DEBUG_BOUNDS 0
#endif
constexpr bool kDebugBounds = VPM_DEBUG_BOUNDS;   // (the Work field it needs is compiled in too)

struct Geo {
    double xw, zw, tx, tz, nx, nz, vx, vz, om;
    double ct, st;                   // cos and sin of the pitch angle
    double cp, sp;                   // cos and sin of pitch + elevator angle (Eqs. 18-20)
    int lev, tev;
};

// Shared-memory workspace of one rollout block (besides the particle and velocity arrays).
struct Work {
    double xg[7];
    double hist[kMaxB + 2];          // previous Gamma_b, previous Gamma_LEV, has_prev flag
    double vt[2 * (2 * kMaxB + 1)];  // relative velocity at collocation then bound points
    double gs[kMaxS];                // Gamma_b, Gamma_LEV, Gamma_TEV of this step
    double fm[3];
    double red[kMaxWarps];
    union {                          // scratch of successive phases of the plate work
        float tgt_f[2 * (kMaxC + kMaxB)];  // plate points in binary32 (binary32 plate sums)
        double b[kMaxS];             // right-hand side of Eq. 10 (active rows; the solve)
        double ld[3 * kMaxB];        // per-panel force x, force z, moment (the loads)
    };
    float bnd_f[4 * kMaxB];          // bound positions as (x_hi, x_lo, z_hi, z_lo)
    float gb_f[kMaxB];               // bound circulations (binary32 copy)
    float4 fresh[2];                 // this step's shed particles before advection (binary32)
    float2 fresh_vel[2];             // and their convection velocities
    Geo geo;
    int n;
    int flag;
    int chunk_next;                  // next unclaimed unit of the pair sums (rows, then diagonals)
    int ndist;                       // 2 while the first two records are the disturbance pair
#if VPM_DEBUG_BOUNDS
    int cap;                         // records the shared arrays hold
#endif
};

// ------------------------------------------------------------------ geometry (the plate warp)

// Plate frame from the glider state. All lanes of the calling warp take part: lane 1 forms sin
// and cos of pitch + elevator angle (needed by the elevator force of Eqs. 18-20 later in the
// step) in the same call in which lane 0 forms those of the pitch angle; lane 0 writes the frame.
__device__ void plate_geometry(const DevParams &p, Work &w)
{
    const int lane = threadIdx.x & 31;
    const double *xg = w.xg;
    double s, c;
    sincos(lane == 1 ? xg[2] + xg[3] : xg[2], &s, &c);
    Geo &G = w.geo;
    if (lane == 1) { G.cp = c; G.sp = s; }
    if (lane == 0) {
        G.ct = c; G.st = s;
        G.xw = xg[0] - p.l_w * c;
        G.zw = xg[1] - p.l_w * s;
        G.tx = -c; G.tz = -s;        // leading edge -> trailing edge
        G.nx = -s; G.nz = c;         // body-up normal
        if (p.fixed_plate) {
            G.vx = 0.0; G.vz = 0.0; G.om = 0.0;
        } else {
            G.vx = xg[4] + p.l_w * xg[6] * s;
            G.vz = xg[5] - p.l_w * xg[6] * c;
            G.om = xg[6];
        }
        if (p.shed_gate == VPM_GATE_OFF) {
            G.lev = G.tev = 1;
        } else {
            double alpha = xg[2] - atan2(G.vz - p.u_inf_z, G.vx - p.u_inf_x);
            alpha = atan2(sin(alpha), cos(alpha));
            int open = fabs(alpha) > p.alpha_crit;
            G.lev = open;
            G.tev = (p.shed_gate != VPM_GATE_BOTH) || open;
        }
    }
    __syncwarp();
}

// Bound vortex j as a double-length binary32 pair (x_hi, x_lo, z_hi, z_lo).
__device__ __forceinline__ void bound_point_f32(const DevParams &p, Work &w, int j)
{
    const Geo &G = w.geo;
    double sj = -0.5 * p.chord + (j + 0.5) * p.lb;
    double bx = G.xw + sj * G.tx, bz = G.zw + sj * G.tz;
    float bxh = (float)bx, bzh = (float)bz;
    w.bnd_f[4 * j + 0] = bxh;
    w.bnd_f[4 * j + 1] = (float)(bx - (double)bxh);
    w.bnd_f[4 * j + 2] = bzh;
    w.bnd_f[4 * j + 3] = (float)(bz - (double)bzh);
}

// Target point t of the plate: collocation points 0..n_c-1, then bound points.
__device__ __forceinline__ void plate_point(const DevParams &p, const Geo &G, int t, double &x,
                                            double &z)
{
    double s = (t < p.n_c) ? (-0.5 * p.chord + t * p.lb)
                           : (-0.5 * p.chord + (t - p.n_c + 0.5) * p.lb);
    x = G.xw + s * G.tx;
    z = G.zw + s * G.tz;
}

// ------------------------------------------------------------------ glider (§III-B)

__device__ void glider_rhs(const DevParams &p, const double *xg, double ct, double st, double cp,
                           double sp, double fwx, double fwz, double mw, double u, double *f)
{
    double xd = xg[4], zd = xg[5], thd = xg[6];
    // elevator velocity (Eq. 18) with phidot = u
    double exd = xd + p.l * thd * st + p.l_e * (thd + u) * sp;
    double ezd = zd - p.l * thd * ct - p.l_e * (thd + u) * cp;
    // flat-plate elevator (Eqs. 19-20): |F_e| = 1/2 rho |v_e|^2 S_e 2 sin(alpha_e) along
    // n_e = (-sin, cos)(th + ph); with alpha_e = th + ph - atan2(zd_e, xd_e),
    // |v_e|^2 sin(alpha_e) = |v_e| (sin(th + ph) xd_e - cos(th + ph) zd_e)
    double vmag = sqrt(exd * exd + ezd * ezd);
    double fe = p.rho * p.s_e * vmag * (sp * exd - cp * ezd);
    double fex = -fe * sp, fez = fe * cp;
    // pitch moment about the centre of gravity with world-frame arms of x_w and x_e
    double wx = -p.l_w * ct, wz = -p.l_w * st;
    double ex = -p.l * ct - p.l_e * cp, ez = -p.l * st - p.l_e * sp;
    double tq = (wx * fwz - wz * fwx) + (ex * fez - ez * fex) + mw;
    f[0] = xd; f[1] = zd; f[2] = thd; f[3] = u;
    f[4] = (fwx + fex) * p.inv_mass;
    f[5] = (fwz + fez) * p.inv_mass - p.g;
    f[6] = tq * p.inv_inertia;
}

// ------------------------------------------------------------------ step phases

// Phase A, binary64 path: wake-induced velocity at the plate points (Eq. 12's sum) and the
// Kelvin sum, by all warps of the block. Each warp takes plate points in turn; its lanes split
// the sources and the partial sums are reduced in binary64. w.red receives one Kelvin partial
// per warp.
template <int KER>
__device__ void plate_sums_f64(const DevParams &p, Work &w, const Part64 *part, int n)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int M = p.n_c + p.n_b;
    for (int t = warp; t < M; t += nwarps) {
        double tx, tz;
        plate_point(p, w.geo, t, tx, tz);
        double su = 0.0, sw = 0.0;
        for (int j = lane; j < n; j += 32) {
            Part64 s = part[j];
            double dx = tx - s.x, dz = tz - s.z;
            double r2 = fma(dx, dx, dz * dz);
            double g = s.g * PairF64<KER>::q(r2, p.rc4, p.inv_rc2);
            su = fma(-dz, g, su);
            sw = fma(dx, g, sw);
        }
        for (int o = 16; o > 0; o >>= 1) {
            su += __shfl_xor_sync(0xffffffffu, su, o);
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
        }
        if (lane == 0) {
            w.vt[2 * t] = su * kInv2Pi;
            w.vt[2 * t + 1] = sw * kInv2Pi;
        }
    }
    double gsum = 0.0;
    for (int j = threadIdx.x; j < n; j += (int)blockDim.x) gsum += part[j].g;
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    if (lane == 0) w.red[warp] = gsum;
}

// Phase A, binary32 path, by the plate warp alone while the other warps start on the pair
// sums. The plate points are formed in binary64 (one lane each) and rounded once; targets then
// go kPlateG at a time so that their dependency chains overlap. Lanes split the sources; the 32
// partial sums of a target are combined by a butterfly in binary32. The Kelvin sum (Eq. 7) is
// Kahan-compensated per lane and combined in binary64; w.red[0] receives it.
constexpr int kPlateG = 4;

template <int KER>
__device__ void plate_sums_f32(const DevParams &p, Work &w, const float4 *part, int n)
{
    const int lane = threadIdx.x & 31;
    const int M = p.n_c + p.n_b;
    const float rc4 = (float)p.rc4, irc2 = (float)p.inv_rc2;
    for (int t = lane; t < M; t += 32) {
        double x, z;
        plate_point(p, w.geo, t, x, z);
        w.tgt_f[2 * t] = (float)x;
        w.tgt_f[2 * t + 1] = (float)z;
    }
    __syncwarp();
    for (int t0 = 0; t0 < M; t0 += kPlateG) {
        float tx[kPlateG], tz[kPlateG], u[kPlateG], v[kPlateG];
#pragma unroll
        for (int g = 0; g < kPlateG; ++g) {
            const int t = min(t0 + g, M - 1);
            tx[g] = w.tgt_f[2 * t];
            tz[g] = w.tgt_f[2 * t + 1];
            u[g] = v[g] = 0.f;
        }
        for (int j = lane; j < n; j += 32) {
            const float4 s = part[j];
#pragma unroll
            for (int g = 0; g < kPlateG; ++g) {
                const float dx = tx[g] - s.x, dz = tz[g] - s.y;
                const float q = s.z * PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
                u[g] = fmaf(-dz, q, u[g]);
                v[g] = fmaf(dx, q, v[g]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int g = 0; g < kPlateG; ++g) {
                u[g] += __shfl_xor_sync(0xffffffffu, u[g], o);
                v[g] += __shfl_xor_sync(0xffffffffu, v[g], o);
            }
        }
        // every lane holds the full sums; lane g converts and scales target t0 + g (binary64
        // instructions cost a full issue slot on the FP64 pipe however few lanes run them)
        float ug = u[0], vg = v[0];
#pragma unroll
        for (int g = 1; g < kPlateG; ++g)
            if (lane == g) { ug = u[g]; vg = v[g]; }
        if (lane < kPlateG && t0 + lane < M) {
            w.vt[2 * (t0 + lane)] = (double)ug * kInv2Pi;
            w.vt[2 * (t0 + lane) + 1] = (double)vg * kInv2Pi;
        }
    }
    float gs = 0.f, gc = 0.f;
    for (int j = lane; j < n; j += 32) kahan_add(gs, gc, part[j].z);
    double gsum = (double)gs - (double)gc;
    for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    if (lane == 0) w.red[0] = gsum;
}

// Pulls lane i's row of this step's inverse surface matrix into L1 while the plate sums run,
// so that the solve's row products do not wait on L2.
__device__ __forceinline__ void prefetch_solve_rows(const DevParams &p, const Geo &G)
{
    const int lane = threadIdx.x & 31, m = p.n_b + G.lev + G.tev;
    const double *ki = p.kinv + (size_t)(G.lev * 2 + G.tev) * kMaxS * kMaxS;
    for (int i = lane; i < m; i += 32)
        for (int j = 0; j < m + 15; j += 16)                 // every 128-byte line of the row
            asm volatile("prefetch.global.L1 [%0];" ::"l"(ki + i * kMaxS + min(j, m - 1)));
}

// Phase B by one warp (all 32 lanes call it): relative velocity at the plate points (Eq. 12),
// the surface solve Gamma_S = K^-1 b (Eq. 11), unsteady Bernoulli loads (Eqs. 13-15), the
// glider's explicit Euler update (Eqs. 18-22) and shedding. Rows of the solve and panels of
// the loads go one per lane; every per-row and per-panel value is formed in the same order as
// a serial evaluation, and the panel loads are summed by lane 0 in panel order. nred is the
// number of Kelvin partials in w.red. Returns the new particle count (all lanes).
template <class R>
__device__ int plate_solve(const DevParams &p, Work &w, typename Store<R>::P *part, int n,
                           double u_ctrl, int nred)
{
    const int lane = threadIdx.x & 31;
    const Geo &G = w.geo;
    const int nb = p.n_b, nc = p.n_c, M = nc + nb;
    // complete Eq. 12: free stream, minus plate translation and rotation e_z x (r_s - r_g)
    for (int t = lane; t < M; t += 32) {
        double x, z;
        plate_point(p, G, t, x, z);
        double rx = x - G.xw, rz = z - G.zw;
        w.vt[2 * t] += p.u_inf_x - G.vx + G.om * rz;
        w.vt[2 * t + 1] += p.u_inf_z - G.vz - G.om * rx;
    }
    __syncwarp();
    // right-hand side of Eq. 10 for the active rows (normal condition, then Kelvin)
    const int lev = G.lev, tev = G.tev, m = nb + lev + tev;
    for (int i = lane; i < nc; i += 32) {
        if ((i == 0 && !lev) || (i == nc - 1 && !tev)) continue;
        w.b[i - (lev ? 0 : 1)] = -(w.vt[2 * i] * G.nx + w.vt[2 * i + 1] * G.nz);
    }
    if (lane == 0) {
        double gw = 0.0;
        for (int i = 0; i < nred; ++i) gw += w.red[i];
        w.b[m - 1] = -gw;
    }
    __syncwarp();
    // Gamma_S = K^-1 b (Eq. 11), one row per lane
    const double *ki = p.kinv + (size_t)(lev * 2 + tev) * kMaxS * kMaxS;
    for (int i = lane; i < m; i += 32) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s = fma(__ldg(ki + i * kMaxS + j), w.b[j], s);
        const int dst = i < nb ? i : (i == nb && lev ? nb : nb + 1);
        w.gs[dst] = s;
    }
    if (lane == 0) {
        if (!lev) w.gs[nb] = 0.0;
        if (!tev) w.gs[nb + 1] = 0.0;
    }
    __syncwarp();
    // unsteady Bernoulli pressure (Eq. 13) and panel loads (Eqs. 14-15), one panel per lane;
    // the running sums of Gamma_b up to the panel are formed as in a serial pass. Each step
    // sheds a new LEV, and all circulation shed at the leading edge counts in the potential
    // jump across the plate, so its time derivative is the new LEV's circulation over dt.
    const bool hp = w.hist[nb + 1] != 0.0;
    const double dlev = hp ? w.gs[nb] * p.inv_dt : 0.0;
    for (int i = lane; i < nb; i += 32) {
        double cum = 0.0, cum_prev = 0.0;
        for (int k = 0; k <= i; ++k) {
            cum += w.gs[k];
            cum_prev += w.hist[k];
        }
        const double *vb = &w.vt[2 * (nc + i)];
        double tang = (w.gs[i] * p.inv_lb) * (vb[0] * G.tx + vb[1] * G.tz);
        double dsum = hp ? (cum - cum_prev) * p.inv_dt : 0.0;
        double dp = p.rho * (tang + dsum + dlev);
        double fx = p.lb * p.span * dp * G.nx, fz = p.lb * p.span * dp * G.nz;
        double si = -0.5 * p.chord + (i + 0.5) * p.lb;
        w.ld[3 * i] = fx;
        w.ld[3 * i + 1] = fz;
        w.ld[3 * i + 2] = (si * G.tx) * fz - (si * G.tz) * fx;
    }
    __syncwarp();
    if (lane == 0) {
        double fwx = 0.0, fwz = 0.0, mw = 0.0;
        for (int i = 0; i < nb; ++i) {
            fwx += w.ld[3 * i];
            fwz += w.ld[3 * i + 1];
            mw += w.ld[3 * i + 2];
        }
        w.fm[0] = fwx; w.fm[1] = fwz; w.fm[2] = mw;
        // glider explicit Euler update with this step's loads
        if (!p.fixed_plate) {
            double f[7];
            glider_rhs(p, w.xg, G.ct, G.st, G.cp, G.sp, fwx, fwz, mw, u_ctrl, f);
            for (int c = 0; c < 7; ++c) w.xg[c] += p.dt * f[c];
        }
        bool finite = isfinite(fwx) && isfinite(fwz) && isfinite(mw);
        for (int c = 0; c < 7; ++c) finite = finite && isfinite(w.xg[c]);
        if (!finite) w.flag |= kStNonFinite;
        w.hist[nb] = w.gs[nb];
        w.hist[nb + 1] = 1.0;
    }
    for (int j = lane; j < nb; j += 32) {
        w.hist[j] = w.gs[j];
        w.gb_f[j] = (float)w.gs[j];
    }
    // W <- W u E (LEV first, then TEV): lane 0 sheds the LEV, lane 1 the TEV
    const double ds = p.shed_dist;
    if ((lane == 0 && lev) || (lane == 1 && tev)) {
        double x, z, g;
        if (lane == 0) {
            plate_point(p, G, 0, x, z);
            x -= ds * G.tx; z -= ds * G.tz; g = w.gs[nb];
        } else {
            plate_point(p, G, nc - 1, x, z);
            x += ds * G.tx; z += ds * G.tz; g = w.gs[nb + 1];
        }
        const int k = lane == 0 ? 0 : lev;
#if VPM_DEBUG_BOUNDS
        if (n + k >= w.cap) {                        // the host's count bound was wrong
            atomicOr(&w.flag, (int)kStCapacity);
        } else
#endif
        {
            part[n + k] = Store<R>::make(x, z, g);
            if constexpr (sizeof(R) == 4) w.fresh[k] = part[n + k];
        }
    }
    __syncwarp();
    return n + lev + tev;
}

// Phase C: convection velocity of every wake particle (Eq. 16) plus the free stream.
//
// Binary32 path. The sum over pairs of particles that existed before this step's shedding
// does not depend on the surface solve, so it runs while the plate warp does the plate work;
// only the bound vortices and the freshly shed vortices need Gamma_S, and their terms are
// added after.
//
// The pair factor of every kernel (Eqs. 4-5, and the Gaussian core) depends on the distance
// alone, and the displacement changes sign when the two particles swap roles, so one
// evaluation of a pair serves both particles' sums. The n old particles form rows of kRow
// (row a: particles kRow a .. kRow a + kRow - 1), and the work comes in two kinds of units:
//   * off-diagonal row a: the row's particles (4 per lane) against every later particle, in
//     blocks of 32 sources (two at a time). A block takes 32 rounds; in round r lane l takes
//     source (l + r) mod 32 for its 4 targets, adds the forward terms to its targets' sums and
//     the reverse terms to the source's running sum, which then moves one lane down. After the
//     32 rounds lane l holds source l's sum over the row's targets and stores it in the block's
//     scratch slot of (row a, source); the targets' compensated sums over the later particles
//     are kept in their own scratch slots;
//   * diagonal group g: kDiagGroup targets against the kRow particles of their own row, every
//     pair in both orders; written to vel.
// Plain sums over 64 sources (two blocks) are added into Kahan-compensated totals. The
// finalize phase adds, per particle, its diagonal sum, its row's forward sum and the reverse
// sums of the earlier rows, in that order. Every partial sum is formed by one warp in a fixed
// order, whichever warp claims it and however many warps the block has.
constexpr int kTile = 64;
#ifndef VPM_SRC_UNROLL
#define VPM_SRC_UNROLL 4      // sources in flight per inner-loop iteration
#endif
constexpr int kSrcUnroll = VPM_SRC_UNROLL;
#ifndef VPM_ROT_UNROLL
#define VPM_ROT_UNROLL 8      // rounds in flight per iteration of the rotation loop (one block;
                              // half as many with two blocks per round)
#endif
constexpr int kRotUnroll = VPM_ROT_UNROLL, kRotUnroll2 = VPM_ROT_UNROLL / 2;
#ifndef VPM_DIAG_UNROLL
#define VPM_DIAG_UNROLL 2     // rounds in flight per iteration of the diagonal unit's block pairs
#endif
#ifndef VPM_DIAG_SELF_UNROLL
#define VPM_DIAG_SELF_UNROLL 3   // and of its in-block rounds (15 of them before the last)
#endif
constexpr int kDiagUnroll = VPM_DIAG_UNROLL, kDiagSelfUnroll = VPM_DIAG_SELF_UNROLL;
constexpr int kRow = 128;     // targets of an off-diagonal row (4 per lane)
// Diagonal units (the pairs among a 128-particle row's own particles). A step with at least
// kDiagPairMin old particles evaluates each such pair once for both particles, one unit per row;
// smaller steps evaluate every pair once per target in groups of 32 DT targets (DT = 1, 2 or 4,
// which give the same bits: each target's sum runs over the row's sources in order). The form
// depends on the particle count alone, so a rollout's result does not depend on the launch
// (block size, DT, batch schedule). Measured with the MPPI batch: fields of 1000-1200 particles
// on 128-thread blocks (72 registers, 7 blocks per SM) run faster with groups of 64 targets,
// fields of 1900-2100 on 256-thread blocks 3 % faster with the once-per-pair units.
#ifndef VPM_DIAG_T
#define VPM_DIAG_T 2          // targets per lane of a per-target diagonal group (1, 2 or 4)
#endif
#ifndef VPM_DIAG_PAIR_MIN
#define VPM_DIAG_PAIR_MIN 1300
#endif
constexpr int kDiagT = VPM_DIAG_T, kDiagPairMin = VPM_DIAG_PAIR_MIN;
// PD (a template flag of the binary32 kernels): the once-per-pair diagonal units are compiled in.
// A launch whose capacity is below kDiagPairMin never needs them (n <= capacity), and leaving
// them out of the 128-thread kernels keeps their row loop's code as fast as without them
// (measured: 4 % on the MPPI batch).


// Sources s0 .. s1-1; targets base + lane + 32 k below lim.
template <int KER, int T>
__device__ __forceinline__ void old_pairs_chunk(const DevParams &p, const float4 *part,
                                                float2 *vel, int s0, int s1, int base, int lim)
{
    const int lane = threadIdx.x & 31;
    const float rc4s = (float)p.rc4, irc2 = (float)p.inv_rc2;
    float tx[T], tz[T], su[T], cu[T], sw[T], cw[T];
#pragma unroll
    for (int k = 0; k < T; ++k) {
        const int i = base + lane + 32 * k;
        const float4 q = part[i < lim ? i : 0];
        tx[k] = q.x;
        tz[k] = q.y;
        su[k] = cu[k] = sw[k] = cw[k] = 0.f;
    }
    for (int j0 = s0; j0 < s1; j0 += kTile) {
        const int je = min(s1, j0 + kTile);
        float au[T], aw[T];
#pragma unroll
        for (int k = 0; k < T; ++k) au[k] = aw[k] = 0.f;
#pragma unroll kSrcUnroll
        for (int j = j0; j < je; ++j) {
            const float4 s = part[j];
#pragma unroll
            for (int k = 0; k < T; ++k) {
                const float dx = tx[k] - s.x, dz = tz[k] - s.y;
                const float g = s.z * PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4s, irc2);
                au[k] = fmaf(-dz, g, au[k]);
                aw[k] = fmaf(dx, g, aw[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < T; ++k) {
            kahan_add(su[k], cu[k], au[k]);
            kahan_add(sw[k], cw[k], aw[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < T; ++k) {
        const int i = base + lane + 32 * k;
        if (i < lim) vel[i] = make_float2(su[k] - cu[k], sw[k] - cw[k]);   // raw, unscaled
    }
}

// Scratch of one block, in float2 slots (sized by the launch's capacity cap, cap32 = cap
// rounded up to 32; an even count, so every block's scratch is 16-byte aligned): the
// Kahan-compensated forward sums of the rows' targets as float4 (u sum, w sum, u compensation,
// w compensation) at [0, 2 cap32), then for each row a < ceil(cap / kRow) - 1 the reverse sums
// of sources kRow (a + 1) .. cap32 - 1.
__host__ __device__ inline long long rev_row_base(int a, int cap32)
{
    return (long long)cap32 * (a + 2) - (long long)(kRow / 2) * a * (a + 1);
}

// Slot of the reverse sum of source j (kRow (a + 1) <= j < cap) over the targets of row a, and
// the float4 index of target i's compensated forward sum (float2 slots 2 i and 2 i + 1).
__host__ __device__ inline long long rev_slot(int a, int j, int cap32)
{
    return rev_row_base(a, cap32) - (long long)kRow * (a + 1) + j;
}
__host__ __device__ inline int fwd_index(int i) { return i; }

__host__ __device__ inline long long rev_slots(int cap)
{
    if (cap <= kRow) return 0;                 // a single row: no off-diagonal work
    const int cap32 = (cap + 31) & ~31, rows = (cap + kRow - 1) / kRow;
    return (rev_row_base(rows - 1, cap32) + 1) & ~1LL;     // even: 16-byte aligned blocks
}

// One block of 32 sources b0 .. b0+31 (all below n when FULL; else the ones at or above n
// take no part) against the 4 targets per lane of an off-diagonal row. On return lane l holds
// the reverse sum of source b0 + l in (ru, rw).
template <int KER, bool FULL>
__device__ __forceinline__ void rotate_block(const DevParams &p, const float4 *part, int n, int b0,
                                             const float (&tx)[4], const float (&tz)[4],
                                             const float (&tg)[4], float (&fu)[4], float (&fw)[4],
                                             float &ru, float &rw)
{
    const int lane = threadIdx.x & 31;
    const float rc4s = (float)p.rc4, irc2 = (float)p.inv_rc2;
    ru = rw = 0.f;
#pragma unroll kRotUnroll
    for (int r = 0; r < 32; ++r) {
        const int j = b0 + ((lane + r) & 31);
        float4 s;
        if (FULL) {
            s = part[j];
        } else {
            s = part[j < n ? j : n - 1];
            if (j >= n) s.z = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s.x, dz = tz[k] - s.y;
            const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4s, irc2);
            const float gs = s.z * q, gt = tg[k] * q;
            fu[k] = fmaf(-dz, gs, fu[k]);
            fw[k] = fmaf(dx, gs, fw[k]);
            ru = fmaf(dz, gt, ru);
            rw = fmaf(-dx, gt, rw);
        }
        ru = __shfl_sync(0xffffffffu, ru, (lane + 1) & 31);
        rw = __shfl_sync(0xffffffffu, rw, (lane + 1) & 31);
    }
}

// Adds the plain sums of the last 64 sources (fu, fw) into the compensated forward sums of row
// a's targets, kept in the block's scratch rather than in registers (the rotation loop needs
// them); `first` starts them from zero.
__device__ __forceinline__ void fold_row(float4 *kst, int a, float (&fu)[4], float (&fw)[4], bool first)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 st = first ? make_float4(0.f, 0.f, 0.f, 0.f) : kst[fwd_index(kRow * a + 32 * k + lane)];
        kahan_add(st.x, st.z, fu[k]);
        kahan_add(st.y, st.w, fw[k]);
        kst[fwd_index(kRow * a + 32 * k + lane)] = st;
        fu[k] = fw[k] = 0.f;
    }
}

// Two full blocks b0 .. b0+31 and b0+32 .. b0+63 at once: each round takes one source of
// each, so two independent running sums travel down the lanes (the chain through the shuffle
// is half as long per pair as with one block). On return lane l holds the reverse sums of
// sources b0 + l (r1) and b0 + 32 + l (r2).
template <int KER>
__device__ __forceinline__ void rotate_two(const DevParams &p, const float4 *part, int b0,
                                           const float (&tx)[4], const float (&tz)[4],
                                           const float (&tg)[4], float (&fu)[4], float (&fw)[4],
                                           float2 &r1, float2 &r2)
{
    const int lane = threadIdx.x & 31;
    const float rc4s = (float)p.rc4, irc2 = (float)p.inv_rc2;
    float ru1 = 0.f, rw1 = 0.f, ru2 = 0.f, rw2 = 0.f;
#pragma unroll kRotUnroll2
    for (int r = 0; r < 32; ++r) {
        const int j = b0 + ((lane + r) & 31);
        const float4 s1 = part[j], s2 = part[j + 32];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s1.x, dz = tz[k] - s1.y;
            const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4s, irc2);
            const float gs = s1.z * q, gt = tg[k] * q;
            fu[k] = fmaf(-dz, gs, fu[k]);
            fw[k] = fmaf(dx, gs, fw[k]);
            ru1 = fmaf(dz, gt, ru1);
            rw1 = fmaf(-dx, gt, rw1);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dx = tx[k] - s2.x, dz = tz[k] - s2.y;
            const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4s, irc2);
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

// Off-diagonal row a (kRow (a + 1) < n, so all of its targets exist).
template <int KER>
__device__ void offdiag_row(const DevParams &p, const float4 *part, float2 *scr, int cap32, int n,
                            int a)
{
    const int lane = threadIdx.x & 31;
    float tx[4], tz[4], tg[4], fu[4], fw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 q = part[kRow * a + 32 * k + lane];
        tx[k] = q.x;
        tz[k] = q.y;
        tg[k] = q.z;
        fu[k] = fw[k] = 0.f;
    }
    float4 *kst = reinterpret_cast<float4 *>(scr);
    float2 *rrow = scr + rev_slot(a, 0, cap32);   // by source index
    int b0 = kRow * (a + 1);                   // a multiple of 64: fold after every two blocks
    bool first = true;
    for (; b0 + 64 <= n; b0 += 64) {
        float2 r1, r2;
        rotate_two<KER>(p, part, b0, tx, tz, tg, fu, fw, r1, r2);
        rrow[b0 + lane] = r1;
        rrow[b0 + 32 + lane] = r2;
        fold_row(kst, a, fu, fw, first);
        first = false;
    }
    if (b0 + 32 <= n) {
        float ru, rw;
        rotate_block<KER, true>(p, part, n, b0, tx, tz, tg, fu, fw, ru, rw);
        rrow[b0 + lane] = make_float2(ru, rw);
        b0 += 32;
    }
    if (b0 < n) {
        float ru, rw;
        rotate_block<KER, false>(p, part, n, b0, tx, tz, tg, fu, fw, ru, rw);
        if (b0 + lane < n) rrow[b0 + lane] = make_float2(ru, rw);
    }
    fold_row(kst, a, fu, fw, first);
}

// One pair of 32-particle blocks of a row's diagonal unit: targets (tx, tz, tg) of block k on
// this lane against source s, forward terms into (fu, fw), reverse terms into the source's
// running sum (ru, rw).
template <int KER>
__device__ __forceinline__ void diag_pair(float rc4s, float irc2, float tx, float tz, float tg,
                                          const float4 &s, float &fu, float &fw, float &ru, float &rw)
{
    const float dx = tx - s.x, dz = tz - s.y;
    const float q = PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4s, irc2);
    const float gs = s.z * q, gt = tg * q;
    fu = fmaf(-dz, gs, fu);
    fw = fmaf(dx, gs, fw);
    ru = fmaf(dz, gt, ru);
    rw = fmaf(-dx, gt, rw);
}

// Diagonal unit of row g with each pair of the row's own particles evaluated once for both
// particles (steps with at least kDiagPairMin particles). Lane l holds particles r0 + 32 k + l of the row's four
// 32-particle blocks k = 0..3 (4 targets per lane, as in offdiag_row). The pairs between blocks
// k < b rotate block b's sources through the lanes as the off-diagonal rows do, with one running
// sum per later block (three); the pairs within a block rotate the block's own sources over 16
// rounds, the 16th on lanes 0-15 only, so that lane l meets l + 16 once. Each particle's diagonal
// sum (its forward terms over both phases, its block's reverse terms, then the reverse terms of
// the earlier blocks, parked in vel) is formed by this warp in a fixed order and written raw to
// vel. FULL: all kRow particles of the row exist; otherwise the missing ones take part with zero
// circulation at a clamped position and nothing is written for them.
template <int KER, bool FULL>
__device__ void diag_row_pairs(const DevParams &p, const float4 *part, float2 *vel, int n, int g)
{
    const int lane = threadIdx.x & 31;
    const int r0 = kRow * g;
    const int nsb = FULL ? 4 : (min(kRow, n - r0) + 31) >> 5;
    const float rc4s = (float)p.rc4, irc2 = (float)p.inv_rc2;
    float tx[4], tz[4], tg[4], fu[4], fw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = r0 + 32 * k + lane;
        const float4 q = part[FULL ? i : min(i, n - 1)];
        tx[k] = q.x;
        tz[k] = q.y;
        tg[k] = (FULL || i < n) ? q.z : 0.f;
        fu[k] = fw[k] = 0.f;
    }
    if (nsb > 1) {
        // blocks b = 1..3 against the targets of the blocks before them
        float ru[3] = {0.f, 0.f, 0.f}, rw[3] = {0.f, 0.f, 0.f};
#pragma unroll kDiagUnroll
        for (int r = 0; r < 32; ++r) {
            const int jl = (lane + r) & 31;
#pragma unroll
            for (int b = 1; b < 4; ++b) {
                if (!FULL && b >= nsb) continue;
                const int j = r0 + 32 * b + jl;
                float4 s = part[FULL ? j : min(j, n - 1)];
                if (!FULL && j >= n) s.z = 0.f;
#pragma unroll
                for (int k = 0; k < b; ++k)
                    diag_pair<KER>(rc4s, irc2, tx[k], tz[k], tg[k], s, fu[k], fw[k], ru[b - 1], rw[b - 1]);
            }
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                ru[b] = __shfl_sync(0xffffffffu, ru[b], (lane + 1) & 31);
                rw[b] = __shfl_sync(0xffffffffu, rw[b], (lane + 1) & 31);
            }
        }
        // lane l now holds the reverse sums of particles r0 + 32 b + l; park them in vel
#pragma unroll
        for (int b = 1; b < 4; ++b) {
            const int i = r0 + 32 * b + lane;
            if (FULL || i < n) vel[i] = make_float2(ru[b - 1], rw[b - 1]);
        }
    }
    // each block with itself: rounds 1..15 on every lane, then round 16 on lanes 0-15
    float su[4] = {0.f, 0.f, 0.f, 0.f}, sw[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll kDiagSelfUnroll
    for (int r = 1; r < 16; ++r) {
        const int jl = (lane + r) & 31;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!FULL && k >= nsb) continue;
            const int j = r0 + 32 * k + jl;
            float4 s = part[FULL ? j : min(j, n - 1)];
            if (!FULL && j >= n) s.z = 0.f;
            diag_pair<KER>(rc4s, irc2, tx[k], tz[k], tg[k], s, fu[k], fw[k], su[k], sw[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            su[k] = __shfl_sync(0xffffffffu, su[k], (lane + 1) & 31);
            sw[k] = __shfl_sync(0xffffffffu, sw[k], (lane + 1) & 31);
        }
    }
    {
        const bool on = lane < 16;
        const int jl = (lane + 16) & 31;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!FULL && k >= nsb) continue;
            const int j = r0 + 32 * k + jl;
            float4 s = part[FULL ? j : min(j, n - 1)];
            if ((!FULL && j >= n) || !on) s.z = 0.f;
            diag_pair<KER>(rc4s, irc2, tx[k], tz[k], on ? tg[k] : 0.f, s, fu[k], fw[k], su[k], sw[k]);
        }
    }
    // lane l holds the in-block reverse sum of particle (l + 16) mod 32 of each block
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        su[k] = __shfl_xor_sync(0xffffffffu, su[k], 16);
        sw[k] = __shfl_xor_sync(0xffffffffu, sw[k], 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = r0 + 32 * k + lane;
        if (!(FULL || i < n)) continue;
        float vx = fu[k] + su[k], vz = fw[k] + sw[k];
        if (k > 0) {
            const float2 c = vel[i];
            vx += c.x;
            vz += c.y;
        }
        vel[i] = make_float2(vx, vz);
    }
}

struct PairPlan {
    int rows_off;   // off-diagonal rows (units 0 .. rows_off - 1, longest first)
    int nunits;     // then the diagonal units: one per row (pair_diag) or groups of 32 DT targets
    bool pair_diag; // n >= kDiagPairMin: each pair of a row's own particles once
};

template <int DT = kDiagT, bool PD = false>
__device__ __forceinline__ PairPlan pair_plan(int n)
{
    PairPlan c;
    const int rows = (n + kRow - 1) / kRow;
    c.rows_off = rows > 1 ? rows - 1 : 0;
    c.pair_diag = PD && n >= kDiagPairMin;
    c.nunits = c.rows_off + (c.pair_diag ? rows : (n + 32 * DT - 1) / (32 * DT));
    return c;
}

// Units are claimed from a counter that is never reset within a rollout: every warp makes
// exactly one failing claim per step, so a step consumes nunits + nwarps claims and every
// thread can track the counter's base for the next step without a barrier.
template <int KER, int DT = kDiagT, bool PD = false>
__device__ void old_pairs_f32(const DevParams &p, Work &w, const float4 *part, float2 *vel,
                              float2 *scr, int cap32, int n, const PairPlan &pp, int claim_base)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int c = 0;
        if (lane == 0) c = atomicAdd(&w.chunk_next, 1) - claim_base;
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= pp.nunits) break;
        if (c < pp.rows_off) {
            offdiag_row<KER>(p, part, scr, cap32, n, c);
        } else if (PD && pp.pair_diag) {
            if constexpr (PD) {
                const int g = c - pp.rows_off;
                if (kRow * (g + 1) <= n) diag_row_pairs<KER, true>(p, part, vel, n, g);
                else diag_row_pairs<KER, false>(p, part, vel, n, g);
            }
        } else {
            const int g = c - pp.rows_off, t0 = 32 * DT * g, r0 = (t0 / kRow) * kRow;
            old_pairs_chunk<KER, DT>(p, part, vel, r0, min(r0 + kRow, n), t0, n);
        }
    }
}

// The old-old sum of target i < n: its diagonal sum (in vel), then its row's forward sum and
// the reverse sums of the earlier rows (scratch). CL: the scratch was written by other CTAs of
// a cluster, so it is read from L2 (ld.global.cg), past this SM's L1. PF: the reverse sums are
// loaded eight at a time before they are added (in the same order), so that a CTA does not wait
// out one L2 latency per row (used by the cluster form: 3 % faster there).
template <bool CL = false, bool PF = false>
__device__ __forceinline__ float2 old_sum(const float2 *vel, const float2 *scr, int cap32,
                                          int rows_off, int i)
{
    const int row = i / kRow;
    float2 v = vel[i];
    if (row == 0 && rows_off == 0) return v;
    float cu = 0.f, cw = 0.f;
    if (row < rows_off) {
        const float4 *fp = reinterpret_cast<const float4 *>(scr) + fwd_index(i);
        float4 f;
        if constexpr (CL) f = __ldcg(fp); else f = *fp;
        kahan_add(v.x, cu, f.x - f.z);
        kahan_add(v.y, cw, f.y - f.w);
    }
    int a = 0;
    if constexpr (PF) {
        for (; a + 8 <= row; a += 8) {
            float2 r8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 *rp = scr + rev_slot(a + j, i, cap32);
                if constexpr (CL) r8[j] = __ldcg(rp); else r8[j] = *rp;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                kahan_add(v.x, cu, r8[j].x);
                kahan_add(v.y, cw, r8[j].y);
            }
        }
    }
    for (; a < row; ++a) {
        const float2 *rp = scr + rev_slot(a, i, cap32);
        float2 r;
        if constexpr (CL) r = __ldcg(rp); else r = *rp;
        kahan_add(v.x, cu, r.x);
        kahan_add(v.y, cw, r.y);
    }
    return make_float2(v.x - cu, v.y - cw);
}

// Bound vortices (singular kernel, Eq. 4) at a target with double-length displacements.
__device__ __forceinline__ void bound_terms_f32(const DevParams &p, const Work &w, float x,
                                                float z, float xl, float zl, float &bu, float &bw)
{
    for (int j = 0; j < p.n_b; ++j) {
        const float dx = (x - w.bnd_f[4 * j]) + (xl - w.bnd_f[4 * j + 1]);
        const float dz = (z - w.bnd_f[4 * j + 2]) + (zl - w.bnd_f[4 * j + 3]);
        const float r2 = fmaf(dx, dx, dz * dz);
        const float q = r2 > 0.f ? __fdividef(w.gb_f[j], r2) : 0.f;
        bu = fmaf(-dz, q, bu);
        bw = fmaf(dx, q, bw);
    }
}

// Full sums of the freshly shed particles n .. n1-1 (at most two; the plate warp, right after
// the solve, while the other warps are still on the old-old pairs), both targets in one pass:
// lanes split the sources, partial sums are combined in binary64, lane f adds the bound terms
// and the free stream for shed particle f.
template <int KER>
__device__ void fresh_velocities_f32(const DevParams &p, Work &w, const float4 *part, int n, int n1)
{
    const int lane = threadIdx.x & 31;
    const int nf = n1 - n;
    if (nf <= 0) return;
    const float rc4 = (float)p.rc4, irc2 = (float)p.inv_rc2;
    const float inv2pi = (float)kInv2Pi;
    const float4 q[2] = {w.fresh[0], w.fresh[nf - 1]};
    float su[2] = {0.f, 0.f}, cu[2] = {0.f, 0.f}, sw[2] = {0.f, 0.f}, cw[2] = {0.f, 0.f};
    for (int j = lane; j < n1; j += 32) {
        const float4 s = part[j];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float dx = q[f].x - s.x, dz = q[f].y - s.y;
            const float g = s.z * PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
            kahan_add(su[f], cu[f], -dz * g);
            kahan_add(sw[f], cw[f], dx * g);
        }
    }
    double du[2], dw[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
        du[f] = (double)su[f] - (double)cu[f];
        dw[f] = (double)sw[f] - (double)cw[f];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            du[f] += __shfl_xor_sync(0xffffffffu, du[f], o);
            dw[f] += __shfl_xor_sync(0xffffffffu, dw[f], o);
        }
    }
    if (lane < nf) {
        const float4 t = lane ? q[1] : q[0];
        const double tu = lane ? du[1] : du[0], tw = lane ? dw[1] : dw[0];
        float xl, zl;
        unpack_lo(t.w, xl, zl);
        float bu = 0.f, bw = 0.f;
        bound_terms_f32(p, w, t.x, t.y, xl, zl, bu, bw);
        w.fresh_vel[lane] = make_float2(fmaf((float)tu + bu, inv2pi, (float)p.u_inf_x),
                                        fmaf((float)tw + bw, inv2pi, (float)p.u_inf_z));
    }
}

// Phase C completion and phase D for one particle: an old target adds the bound terms and the
// freshly shed vortices (from their pre-advection copies) to its old-old sum; every particle is
// then advected by explicit Euler (double-length positions) and decayed exactly,
// Gamma <- Gamma exp(-gamma dt) (Eq. 17). The record is read and written by the thread that
// owns it, so no barrier separates the velocity from the advection. `bad` collects non-finite
// velocities. CL (a CTA of a cluster that runs one rollout): the scratch is read from L2 and
// the advected record is written into the field of every CTA of the cluster.
template <int KER, bool CL = false, bool PF = false>
__device__ __forceinline__ void finalize_one(const DevParams &p, const Work &w, float4 *part,
                                             const float2 *vel, const float2 *scr, int cap32,
                                             int rows_off, int n, int nf, int i, double *probe_vel,
                                             bool &bad)
{
    const float rc4 = (float)p.rc4, irc2 = (float)p.inv_rc2;
    const float inv2pi = (float)kInv2Pi;
    const float uix = (float)p.u_inf_x, uiz = (float)p.u_inf_z;
    const float dth = (float)p.dt, dtl = (float)(p.dt - (double)dth);
    const float dch = (float)p.decay, dcl = (float)(p.decay - (double)dch);
    float4 q;
    float2 v;
    float xl, zl;
    if (i < n) {
        q = part[i];
        const float2 raw = old_sum<CL, PF>(vel, scr, cap32, rows_off, i);
        unpack_lo(q.w, xl, zl);
        float bu = 0.f, bw = 0.f;
        bound_terms_f32(p, w, q.x, q.y, xl, zl, bu, bw);
        for (int f = 0; f < nf; ++f) {
            const float4 s = w.fresh[f];
            const float dx = q.x - s.x, dz = q.y - s.y;
            const float g = s.z * PairF32<KER>::q(fmaf(dx, dx, dz * dz), rc4, irc2);
            bu = fmaf(-dz, g, bu);
            bw = fmaf(dx, g, bw);
        }
        v = make_float2(fmaf(raw.x + bu, inv2pi, uix), fmaf(raw.y + bw, inv2pi, uiz));
    } else {
        q = w.fresh[i - n];
        v = w.fresh_vel[i - n];
        unpack_lo(q.w, xl, zl);
    }
    if (probe_vel) { probe_vel[2 * i] = v.x; probe_vel[2 * i + 1] = v.y; }
    bad |= !(isfinite(v.x) && isfinite(v.y));
    const float ddx = fmaf(v.x, dth, fmaf(v.x, dtl, xl));
    const float ddz = fmaf(v.y, dth, fmaf(v.y, dtl, zl));
    float sx, ex, sz, ez;
    two_sum(q.x, ddx, sx, ex);
    two_sum(q.y, ddz, sz, ez);
    q.x = sx;
    q.y = sz;
    q.z = fmaf(q.z, dcl, q.z * dch);
    q.w = pack_lo(ex, ez);
    if constexpr (CL) {
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        const int C = (int)cl.num_blocks();
        for (int r = 0; r < C; ++r) *cl.map_shared_rank(part + i, r) = q;
    } else {
        part[i] = q;
    }
}

// Phase C completion and phase D for every particle of the step, by the whole block (PF: see
// old_sum).
template <int KER, bool PF = false>
__device__ void finalize_advect_f32(const DevParams &p, Work &w, float4 *part, const float2 *vel,
                                    const float2 *scr, int cap32, int rows_off, int n, int n1,
                                    double *probe_vel)
{
    const int nf = n1 - n;
    bool bad = false;
    for (int i = threadIdx.x; i < n1; i += (int)blockDim.x)
        finalize_one<KER, false, PF>(p, w, part, vel, scr, cap32, rows_off, n, nf, i, probe_vel, bad);
    if (bad) atomicOr(&w.flag, (int)kStNonFinite);
}

// Convection velocity (Eq. 16) of one target at (x, z) on the binary64 path, by one warp: lane l
// sums sources l, l + 32, ... in order, lanes below n_b add bound vortex l, and a butterfly
// combines the 32 partial sums (every lane ends with the same bits). Binary64 warp instructions
// take the same time however many lanes are active, so a warp per target keeps every lane busy
// even when a block has few targets; the one-block and the cluster paths both use this order.
template <int KER>
__device__ __forceinline__ double2 convect_target_f64(const DevParams &p, const Work &w,
                                                      const Part64 *part, int n1, double x,
                                                      double z)
{
    const int lane = threadIdx.x & 31;
    const Geo &G = w.geo;
    double su = 0.0, sw = 0.0;
    for (int j = lane; j < n1; j += 32) {
        const Part64 s = part[j];
        const double dx = x - s.x, dz = z - s.z;
        const double g = s.g * PairF64<KER>::q(fma(dx, dx, dz * dz), p.rc4, p.inv_rc2);
        su = fma(-dz, g, su);
        sw = fma(dx, g, sw);
    }
    if (lane < p.n_b) {
        const double sj = -0.5 * p.chord + (lane + 0.5) * p.lb;
        const double dx = x - (G.xw + sj * G.tx), dz = z - (G.zw + sj * G.tz);
        const double r2 = fma(dx, dx, dz * dz);
        const double q = r2 > 0.0 ? w.gs[lane] / r2 : 0.0;
        su = fma(-dz, q, su);
        sw = fma(dx, q, sw);
    }
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    return make_double2(su * kInv2Pi + p.u_inf_x, sw * kInv2Pi + p.u_inf_z);
}

// Phase C on the binary64 path: one warp per target.
template <int KER>
__device__ void convect_f64(const DevParams &p, const Work &w, const Part64 *part, double2 *vel,
                            int n, double *probe_vel)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int i = warp; i < n; i += nwarps) {
        const Part64 pi = part[i];
        const double2 v = convect_target_f64<KER>(p, w, part, n, pi.x, pi.z);
        if (lane == 0) {
            vel[i] = v;
            if (probe_vel) { probe_vel[2 * i] = v.x; probe_vel[2 * i + 1] = v.y; }
        }
    }
}

// Phase D on the binary64 path: explicit Euler advection and the exact decay of Eq. 17.
__device__ void advect_f64(const DevParams &p, Work &w, Part64 *part, const double2 *vel, int n)
{
    bool bad = false;
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) {
        Part64 q = part[i];
        const double2 v = vel[i];
        bad |= !(isfinite(v.x) && isfinite(v.y));
        q.x += p.dt * v.x;
        q.z += p.dt * v.y;
        q.g *= p.decay;
        part[i] = q;
    }
    if (bad) atomicOr(&w.flag, (int)kStNonFinite);
}

// Merging (§III-A): while N > N_w,max the two oldest wake particles become one at their mean
// position with the summed circulation; the merged particle stays the oldest. The first d
// records (the disturbance pair, if present) are not part of the wake budget and are left
// alone. Applying it m = N - d - N_w,max times merges records d..d+m in order and shifts the
// rest down by m.
// Kept out of line, as is terminate_pair: inlined into the step, these rarely-taken paths
// changed the code generated for the pair loop and cost 15 % on large fields (measured).
template <class R>
__device__ __noinline__ int merge_oldest(const DevParams &p, typename Store<R>::P *part, int n, int d)
{
    using P = typename Store<R>::P;
    if (p.n_wake_max <= 0 || n - d <= p.n_wake_max) return n;
    const int m = n - d - p.n_wake_max;
    __shared__ P s_merged;
    if (threadIdx.x == 0) {
        double x, z;
        Store<R>::xz(part[d], x, z);
        double g = Store<R>::gam(part[d]);
        for (int q = 1; q <= m; ++q) {
            double x2, z2;
            Store<R>::xz(part[d + q], x2, z2);
            x = 0.5 * (x + x2);
            z = 0.5 * (z + z2);
            g = g + Store<R>::gam(part[d + q]);
        }
        s_merged = Store<R>::make(x, z, g);
    }
    __syncthreads();
    const int nn = n - m;
    for (int base = d + 1; base < nn; base += (int)blockDim.x) {
        const int i = base + threadIdx.x;
        P tmp;
        if (i < nn) tmp = part[i + m];
        __syncthreads();
        if (i < nn) part[i] = tmp;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[d] = s_merged;
    __syncthreads();
    return nn;
}

// Disturbance termination (§V): with the plate at its updated position, the pair in records 0
// and 1 is removed once the segment joining it crosses the chord line (leading to trailing
// collocation point) moved by 2 % of the chord against the normal. A crossing needs each
// segment's ends strictly on opposite sides of the other's line (signed areas, binary64).
__device__ __forceinline__ double side_of(double ax, double az, double bx, double bz, double px,
                                          double pz)
{
    return (bx - ax) * (pz - az) - (bz - az) * (px - ax);
}

template <class R>
__device__ __noinline__ int terminate_pair(const DevParams &p, Work &w, typename Store<R>::P *part, int n)
{
    __shared__ int s_cross;
    if (threadIdx.x == 0) {
        int cross = 0;
        if (n >= 2) {
            double x0, z0, x1, z1;
            Store<R>::xz(part[0], x0, z0);
            Store<R>::xz(part[1], x1, z1);
            double sn, cs;
            sincos(w.xg[2], &sn, &cs);
            const double xw = w.xg[0] - p.l_w * cs, zw = w.xg[1] - p.l_w * sn;
            const double tx = -cs, tz = -sn, nx = -sn, nz = cs, off = 0.02 * p.chord;
            const double s0 = -0.5 * p.chord, s1 = -0.5 * p.chord + p.n_b * p.lb;
            const double ax = xw + s0 * tx - off * nx, az = zw + s0 * tz - off * nz;
            const double bx = xw + s1 * tx - off * nx, bz = zw + s1 * tz - off * nz;
            const double o1 = side_of(ax, az, bx, bz, x0, z0), o2 = side_of(ax, az, bx, bz, x1, z1);
            const double o3 = side_of(x0, z0, x1, z1, ax, az), o4 = side_of(x0, z0, x1, z1, bx, bz);
            cross = ((o1 > 0.0 && o2 < 0.0) || (o1 < 0.0 && o2 > 0.0)) &&
                    ((o3 > 0.0 && o4 < 0.0) || (o3 < 0.0 && o4 > 0.0));
        }
        s_cross = cross;
    }
    __syncthreads();
    if (!s_cross) return n;
    using P = typename Store<R>::P;
    for (int base = 0; base < n - 2; base += (int)blockDim.x) {
        const int i = base + threadIdx.x;
        P tmp;
        if (i < n - 2) tmp = part[i + 2];
        __syncthreads();
        if (i < n - 2) part[i] = tmp;
        __syncthreads();
    }
    if (threadIdx.x == 0) w.ndist = 0;
    __syncthreads();
    return n - 2;
}

// The warp that does the binary32 path's plate work: it varies with the block (block index mod
// warps per block). Measured against always using warp 0: 2.5 % faster on the MPPI batch and
// 5 % slower on the perch-shape batch (<= 62 particles); a variant that chose by field size
// (varying above 256 particles, warp 0 below) was fast on the perch shape but lost the gain on
// the MPPI batch, where it chose the same warps. The pair loop's code generation is this
// sensitive to the surrounding code, so the form kept is the one that measures best on the
// MPPI batch.
__device__ __forceinline__ int plate_warp()
{
    return (int)(blockIdx.x & ((blockDim.x >> 5) - 1));
}

// One full step of one rollout. All threads call it with the same particle count n (updated
// here) and unit-claim base; returns with the block synchronised.
template <class R, int KER, int DT = kDiagT, bool PD = false>
__device__ void step_once(const DevParams &p, Work &w, typename Store<R>::P *part,
                          typename Store<R>::V *vel, double u_ctrl, const RolloutArgs &a,
                          bool probe, int &n, int &claim_base)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    int n1;
    if constexpr (sizeof(R) == 4) {
        // the plate warp: plate geometry, plate sums, surface solve, loads, glider, shedding
        // and the shed particles' velocities; meanwhile (and afterwards for the plate warp)
        // every warp works on the old-old pair sums
        if (warp == plate_warp()) {
            const int lane = tid & 31;
            plate_geometry(p, w);
            prefetch_solve_rows(p, w.geo);
            if (lane < p.n_b) bound_point_f32(p, w, lane);
            plate_sums_f32<KER>(p, w, part, n);
            __syncwarp();
            const int m = plate_solve<R>(p, w, part, n, u_ctrl, 1);
            if (lane == 0) w.n = m;
            fresh_velocities_f32<KER>(p, w, part, n, m);
        }
        const PairPlan pp = pair_plan<DT, PD>(n);
        const int cap32 = (a.cap + 31) & ~31;
        float2 *scr = a.rev ? a.rev + (size_t)blockIdx.x * a.rev_stride : nullptr;
#if VPM_DEBUG_BOUNDS
        if (pp.rows_off > 0 && (!scr || a.rev_stride < rev_slots(a.cap) || n > a.cap)) {
            if (tid == 0) atomicOr(&w.flag, (int)kStCapacity);   // the host's scratch was short
            __syncthreads();
            return;
        }
#endif
        old_pairs_f32<KER, DT, PD>(p, w, part, vel, scr, cap32, n, pp, claim_base);
        claim_base += pp.nunits + (int)(blockDim.x >> 5);
        __syncthreads();
        n1 = w.n;
        if (probe) {
            const int M = p.n_c + p.n_b;
            if (a.probe_vt) for (int t = tid; t < 2 * M; t += (int)blockDim.x) a.probe_vt[t] = w.vt[t];
            if (a.probe_gs) for (int t = tid; t < p.n_b + 2; t += (int)blockDim.x) a.probe_gs[t] = w.gs[t];
            if (a.probe_fm && tid < 3) a.probe_fm[tid] = w.fm[tid];
        }
        // (the reverse-sum loads eight at a time, PF, measured here: 1.8 % slower on the
        // ~2000-particle fields, no change on one block of 8000; the cluster form keeps it)
        finalize_advect_f32<KER>(p, w, part, vel, scr, cap32, pp.rows_off, n, n1,
                                 probe ? a.probe_vel : nullptr);
    } else {
        if (warp == 0) plate_geometry(p, w);
        __syncthreads();
        plate_sums_f64<KER>(p, w, part, n);
        __syncthreads();
        if (warp == 0) {
            const int m = plate_solve<R>(p, w, part, n, u_ctrl, (int)(blockDim.x >> 5));
            if (tid == 0) w.n = m;
        }
        __syncthreads();
        n1 = w.n;
        convect_f64<KER>(p, w, part, vel, n1, probe ? a.probe_vel : nullptr);
        if (probe) {
            const int M = p.n_c + p.n_b;
            if (a.probe_vt) for (int t = tid; t < 2 * M; t += (int)blockDim.x) a.probe_vt[t] = w.vt[t];
            if (a.probe_gs) for (int t = tid; t < p.n_b + 2; t += (int)blockDim.x) a.probe_gs[t] = w.gs[t];
            if (a.probe_fm && tid < 3) a.probe_fm[tid] = w.fm[tid];
        }
        __syncthreads();
        advect_f64(p, w, part, vel, n1);
    }
    __syncthreads();
    if (w.ndist == 2) n1 = terminate_pair<R>(p, w, part, n1);
    n = merge_oldest<R>(p, part, n1, w.ndist);
}

template <class R>
__device__ void load_state(const RolloutArgs &a, Work &w, typename Store<R>::P *part, int rid)
{
    using P = typename Store<R>::P;
    const long long off = a.root_offset ? a.root_offset[rid] : (long long)rid * a.root_stride;
    const P *rp = static_cast<const P *>(a.root_part) + off;
    const int n = a.root_n[(a.root_stride || a.root_offset) ? rid : 0];
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) part[i] = rp[i];
    const double *g = a.x0 ? a.x0 + (size_t)rid * 7 : a.root_glider + (size_t)rid * a.state_stride;
    const double *h = a.root_hist + (size_t)rid * a.state_stride;
    if (threadIdx.x < 7) w.xg[threadIdx.x] = g[threadIdx.x];
    if (threadIdx.x < a.p.n_b + 2) w.hist[threadIdx.x] = h[threadIdx.x];
    if (threadIdx.x == 0) {
        w.n = n; w.flag = 0; w.chunk_next = 0;
        w.ndist = a.root_ndist ? a.root_ndist[(a.root_stride || a.root_offset) ? rid : 0] : 0;
#if VPM_DEBUG_BOUNDS
        w.cap = a.cap;
#endif
    }
    __syncthreads();
}

template <class R>
__device__ void store_state(const RolloutArgs &a, Work &w, const typename Store<R>::P *part,
                            int rid)
{
    using P = typename Store<R>::P;
    P *op = static_cast<P *>(a.out_part) + (size_t)rid * a.out_stride;
    const int n = w.n;
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) op[i] = part[i];
    double *g = a.out_glider + (size_t)rid * a.out_state_stride;
    double *h = a.out_hist + (size_t)rid * a.out_state_stride;
    if (threadIdx.x < 7) g[threadIdx.x] = w.xg[threadIdx.x];
    if (threadIdx.x < a.p.n_b + 2) h[threadIdx.x] = w.hist[threadIdx.x];
    if (threadIdx.x == 0) a.out_n[a.out_stride ? rid : 0] = n;
    if (threadIdx.x == 0 && a.out_ndist) a.out_ndist[a.out_stride ? rid : 0] = w.ndist;
}

template <class R>
__device__ void finish(const RolloutArgs &a, Work &w, const typename Store<R>::P *part, int rid)
{
    const DevParams &p = a.p;
    const int n = w.n;
    if (threadIdx.x == 0) {
        double J = 0.0;
        for (int c = 0; c < 7; ++c) {
            double d = w.xg[c] - p.x_d[c];
            J += d * p.q[c] * d;
        }
        if (!isfinite(J)) w.flag |= kStNonFinite;
        if (a.costs) a.costs[rid] = w.flag ? __int_as_float(0x7fc00000) : (float)J;
        if (w.flag && a.status) atomicOr(a.status, w.flag);
        if (a.count) a.count[rid] = n;
    }
    if (a.final_glider && threadIdx.x < 7) a.final_glider[rid * 7 + threadIdx.x] = w.xg[threadIdx.x];
    if (a.field) {
        double *f = a.field + (size_t)rid * a.field_cap * 3;
        for (int i = threadIdx.x; i < n; i += (int)blockDim.x) {
            double x, z;
            Store<R>::xz(part[i], x, z);
            f[3 * i] = x;
            f[3 * i + 1] = z;
            f[3 * i + 2] = Store<R>::gam(part[i]);
        }
    }
}

// Pacing of the blocks that share an SM. All blocks of a one-wave launch start together, but
// the warp schedulers favour the oldest warps, so left alone the first of seven co-resident
// blocks finishes after about 56 % of the launch and the last runs alone at its end, where one
// block's warps cannot hide the latency of the pair loop's shuffles (measured: 66 % of the
// SM's rate with one block). A block that is more than kPaceAhead steps ahead of the slowest
// block on its SM therefore sleeps until that block catches up, for at most kPaceWaits short
// sleeps per step; giving up only costs time, never changes a result. Blocks more than
// kPaceWindow steps behind are not waited for: such a block started late (other work held its
// SM when the launch began) and cannot catch up.
constexpr int kPaceSlots = 8, kPaceAhead = 1, kPaceWaits = 1000, kPaceWindow = 4;
constexpr int kPaceSms = 1024;    // SM ids paced (blocks on an SM with a larger id are not)
// Fields that stay small have short, plate-bound steps (~18 us at 60 particles), where a
// 1 us sleep and the extra barrier cost more than the tail they remove: pacing is for launches
// whose fields can exceed this many particles (measured: the perch-shape batch of 1024 took
// 2.64 ms paced against 2.30 ms unpaced).
// Pacing is off unless the environment variable VPM_PACE is 1 when a launch is made. With the
// current pair phase it no longer pays on the MPPI batch (K = 1024, H = 100: 36.8 ms paced
// against 36.3 ms unpaced), but its code stays in the kernel: removing it changed the row loop's
// register allocation and cost 2.4 % (37.7 ms).
constexpr int kPaceMinCap = 256;

static bool pacing_requested()
{
    const char *e = getenv("VPM_PACE");
    return e && e[0] == '1' && e[1] == 0;
}

__device__ __forceinline__ unsigned sm_id()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Thread 0: takes a slot on this SM (-1: pacing off for this block).
__device__ int pace_join(const RolloutArgs &a, unsigned sm)
{
    if (!a.pace_mask || sm >= (unsigned)a.pace_sms) return -1;
    for (int b = 0; b < kPaceSlots; ++b) {
        const unsigned old = atomicOr(&a.pace_mask[sm], 1u << b);
        if (!(old & (1u << b))) {
            atomicExch(&a.pace_prog[sm * kPaceSlots + b], 0);
            return b;
        }
    }
    return -1;
}

// Thread 0, before step k: publishes k and waits while the block is ahead.
__device__ void pace_step(const RolloutArgs &a, unsigned sm, int slot, int k)
{
    int *prog = a.pace_prog + sm * kPaceSlots;
    atomicExch(&prog[slot], k);
    for (int it = 0; it < kPaceWaits; ++it) {
        const unsigned m = atomicOr(&a.pace_mask[sm], 0u);
        int lo = INT_MAX;
        for (int b = 0; b < kPaceSlots; ++b) {
            if (b == slot || !(m & (1u << b))) continue;
            const int pb = atomicOr(&prog[b], 0);
            if (pb >= k - kPaceWindow) lo = min(lo, pb);
        }
        if (lo == INT_MAX || k <= lo + kPaceAhead) return;
        __nanosleep(1000);
    }
}

// One rollout of a.H steps by the whole block, field resident in shared memory.
template <class R, int KER, int DT = kDiagT, bool PD = false>
__device__ void run_rollout(const RolloutArgs &a, Work &w, typename Store<R>::P *part,
                            typename Store<R>::V *vel, int rid)
{
    load_state<R>(a, w, part, rid);
    int n = w.n, claim_base = 0;
    __shared__ int s_slot;
    const unsigned sm = sm_id();
    if (threadIdx.x == 0) s_slot = pace_join(a, sm);
    __syncthreads();
    const int slot = s_slot;
    for (int k = 0; k < a.H; ++k) {
        if (slot >= 0 && k > 0) {
            if (threadIdx.x == 0) pace_step(a, sm, slot, k);
            __syncthreads();
        }
        double u = a.controls ? (double)a.controls[(size_t)rid * a.ctrl_stride + a.step0 + k]
                              : a.u_const;
        if (a.pol_gains && (int)(threadIdx.x >> 5) == (sizeof(R) == 4 ? plate_warp() : 0)) {
            // the feedback control from the glider state in shared memory, formed by the warp
            // that does the plate work, the only warp that uses the control
            const size_t j = (size_t)a.pol_offset + k;
            double fb = (double)a.pol_ubar[j];
            for (int c = 0; c < 7; ++c)
                fb -= a.pol_gains[j * 7 + c] * (w.xg[c] - a.pol_xbar[j * 7 + c]);
            u = (a.controls ? u : 0.0) + fb;
        }
        step_once<R, KER, DT, PD>(a.p, w, part, vel, u, a, a.H == 1, n, claim_base);
        if (a.traj && threadIdx.x < 7)
            a.traj[((size_t)rid * a.H + k) * 7 + threadIdx.x] = w.xg[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        w.n = n;
        if (slot >= 0) atomicAnd(&a.pace_mask[sm], ~(1u << slot));   // leaves the SM's pacing
    }
    __syncthreads();
    if (a.out_part) store_state<R>(a, w, part, rid);
    finish<R>(a, w, part, rid);
}

#ifndef VPM_MIN_BLOCKS
#define VPM_MIN_BLOCKS 7      // 7 blocks of 128 threads per SM: 1024 rollouts of ~1200 particles in one wave
#endif

// Register budget per block size: 128 threads keep 7 blocks per SM; larger blocks serve large
// fields, whose shared memory allows 1-3 blocks per SM anyway.
__host__ __device__ constexpr int min_blocks_for(int nt)
{
    return nt <= 128 ? VPM_MIN_BLOCKS : (nt <= 256 ? 3 : 1);
}

// K rollouts (blockIdx.x + rid0 = rollout), H steps each.
template <class R, int KER, int NT, bool PD>
__global__ void __launch_bounds__(NT, min_blocks_for(NT)) rollout_kernel(const RolloutArgs a)
{
    using P = typename Store<R>::P;
    using V = typename Store<R>::V;
    extern __shared__ __align__(16) unsigned char smem[];
    P *part = reinterpret_cast<P *>(smem);
    V *vel = reinterpret_cast<V *>(smem + sizeof(P) * (size_t)a.cap);
    __shared__ Work w;
    run_rollout<R, KER, kDiagT, PD>(a, w, part, vel, blockIdx.x + a.rid0);
}

// Persistent form for batches of uneven rollouts: each block claims the next rollout of
// a.order until all a.n_items are done. Which block runs a rollout does not change its result.
template <class R, int KER, int NT, int DT = kDiagT, bool PD = true>
__global__ void __launch_bounds__(NT, min_blocks_for(NT)) uneven_kernel(const RolloutArgs a)
{
    using P = typename Store<R>::P;
    using V = typename Store<R>::V;
    extern __shared__ __align__(16) unsigned char smem[];
    P *part = reinterpret_cast<P *>(smem);
    V *vel = reinterpret_cast<V *>(smem + sizeof(P) * (size_t)a.cap);
    __shared__ Work w;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int q = s_item;
        __syncthreads();
        if (q >= a.n_items) break;
        run_rollout<R, KER, DT, PD>(a, w, part, vel, a.order[q]);
    }
}

// ------------------------------------------------------------------ binary32 rollouts over a cluster

// One binary32 rollout spread over a thread-block cluster of C CTAs (2 or 4; a schedule of the
// uneven batch for large fields). Every CTA holds the whole field in its shared memory and runs
// the plate warp's serial work (geometry, plate sums, solve, loads, glider, shedding) from
// identical data, so every CTA has the same plate state, particle count and shed particles.
// The step's pair units are split by index: unit u goes to CTA u mod C, and the CTA's warps claim
// its units in order. Rows write their partial sums to the cluster's scratch in global memory;
// diagonal units write their targets' sums into their CTA's vel. After a cluster barrier (release
// and acquire at cluster scope) a particle is completed and advected by the CTA that ran its
// diagonal unit (the freshly shed particles by CTA 0), which writes the new record into the field
// of every CTA through distributed shared memory; a second cluster barrier ends the step, and
// termination and merging then run on every CTA from identical fields. Every partial sum is
// formed by one warp in the same order as on the one-CTA path and combined per particle in the
// same order, so the results are the same bits whatever C.
template <int KER, int DT>
__device__ void old_pairs_f32_cl(const DevParams &p, Work &w, const float4 *part, float2 *vel,
                                 float2 *scr, int cap32, int n, const PairPlan &pp, int claim_base,
                                 int rank, int C, int nl)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int li = 0;
        if (lane == 0) li = atomicAdd(&w.chunk_next, 1) - claim_base;
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= nl) break;
        const int c = rank + C * li;
        if (c < pp.rows_off) {
            offdiag_row<KER>(p, part, scr, cap32, n, c);
        } else if (pp.pair_diag) {
            const int g = c - pp.rows_off;
            if (kRow * (g + 1) <= n) diag_row_pairs<KER, true>(p, part, vel, n, g);
            else diag_row_pairs<KER, false>(p, part, vel, n, g);
        } else {
            const int g = c - pp.rows_off, t0 = 32 * DT * g, r0 = (t0 / kRow) * kRow;
            old_pairs_chunk<KER, DT>(p, part, vel, r0, min(r0 + kRow, n), t0, n);
        }
    }
}

template <int KER, int DT>
__device__ void step_once_cl(const DevParams &p, Work &w, float4 *part, float2 *vel, double u_ctrl,
                             const RolloutArgs &a, float2 *scr, int rank, int C, int &n,
                             int &claim_base)
{
    namespace cg = cooperative_groups;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == plate_warp()) {
        const int lane = tid & 31;
        plate_geometry(p, w);
        prefetch_solve_rows(p, w.geo);
        if (lane < p.n_b) bound_point_f32(p, w, lane);
        plate_sums_f32<KER>(p, w, part, n);
        __syncwarp();
        const int m = plate_solve<float>(p, w, part, n, u_ctrl, 1);
        if (lane == 0) w.n = m;
        fresh_velocities_f32<KER>(p, w, part, n, m);
    }
    const PairPlan pp = pair_plan<DT, true>(n);
    const int cap32 = (a.cap + 31) & ~31;
    const int nl = pp.nunits > rank ? (pp.nunits - rank + C - 1) / C : 0;
    old_pairs_f32_cl<KER, DT>(p, w, part, vel, scr, cap32, n, pp, claim_base, rank, C, nl);
    claim_base += nl + (int)(blockDim.x >> 5);
    cg::this_cluster().sync();       // every CTA's partial sums written; plate results in place
    int n1 = w.n;
    const int nf = n1 - n, gsz = pp.pair_diag ? kRow : 32 * DT;
    bool bad = false;
    for (int i = tid; i < n1; i += (int)blockDim.x) {
        const int owner = i < n ? (pp.rows_off + i / gsz) % C : 0;
        if (owner == rank)
            finalize_one<KER, true, true>(p, w, part, vel, scr, cap32, pp.rows_off, n, nf, i, nullptr, bad);
    }
    if (bad) atomicOr(&w.flag, (int)kStNonFinite);
    cg::this_cluster().sync();       // the advected field is complete in every CTA
    if (w.ndist == 2) n1 = terminate_pair<float>(p, w, part, n1);
    n = merge_oldest<float>(p, part, n1, w.ndist);
}

template <int KER, int DT>
__device__ void run_rollout_cl(const RolloutArgs &a, Work &w, float4 *part, float2 *vel, float2 *scr,
                               int rid, int rank, int C)
{
    namespace cg = cooperative_groups;
    load_state<float>(a, w, part, rid);
    int n = w.n, claim_base = 0;
    for (int k = 0; k < a.H; ++k) {
        double u = a.controls ? (double)a.controls[(size_t)rid * a.ctrl_stride + a.step0 + k]
                              : a.u_const;
        if (a.pol_gains && (int)(threadIdx.x >> 5) == plate_warp()) {
            const size_t j = (size_t)a.pol_offset + k;
            double fb = (double)a.pol_ubar[j];
            for (int c = 0; c < 7; ++c)
                fb -= a.pol_gains[j * 7 + c] * (w.xg[c] - a.pol_xbar[j * 7 + c]);
            u = (a.controls ? u : 0.0) + fb;
        }
        step_once_cl<KER, DT>(a.p, w, part, vel, u, a, scr, rank, C, n, claim_base);
        if (rank == 0 && a.traj && threadIdx.x < 7)
            a.traj[((size_t)rid * a.H + k) * 7 + threadIdx.x] = w.xg[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        w.n = n;
        if (rank != 0 && w.flag) atomicOr(cg::this_cluster().map_shared_rank(&w.flag, 0), w.flag);
    }
    cg::this_cluster().sync();
    if (rank == 0) {
        if (a.out_part) store_state<float>(a, w, part, rid);
        finish<float>(a, w, part, rid);
    }
}

// Persistent cluster form of uneven_kernel: CTA 0 of each cluster claims the next rollout of
// a.order (without an order, rollout a.rid0 + claim) and hands its index to the other CTAs; the
// cluster's scratch is slot blockIdx.x / C.
template <int KER, int NT, int DT>
__global__ void __launch_bounds__(NT, min_blocks_for(NT)) uneven_cluster_kernel(const RolloutArgs a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *part = reinterpret_cast<float4 *>(smem);
    float2 *vel = reinterpret_cast<float2 *>(smem + sizeof(float4) * (size_t)a.cap);
    __shared__ Work w;
    __shared__ int s_item;
    float2 *scr = a.rev ? a.rev + (size_t)(blockIdx.x / C) * a.rev_stride : nullptr;
    cl.sync();                       // every CTA of the cluster has started before any remote write
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int q = atomicAdd(a.counter, 1);
            for (int r = 0; r < C; ++r) *cl.map_shared_rank(&s_item, r) = q;
        }
        cl.sync();
        const int q = s_item;
        if (q >= a.n_items) break;
        run_rollout_cl<KER, DT>(a, w, part, vel, scr, a.order ? a.order[q] : a.rid0 + q, rank, C);
        cl.sync();                   // every CTA is done with this rollout and with s_item
    }
}

// ------------------------------------------------------------------ host-side launch helpers

// Raises a kernel's dynamic shared-memory limit to at least smem, once per size increase (the
// 48 KB default covers static + dynamic, so launchers always opt in; the library runs on one
// device per process). Host threads may launch at the same time (the NMPC planner and control
// paths, the serving worker), so the raise happens under a lock and the limit only grows.
static std::mutex g_grant_mutex;

template <class F>
static cudaError_t grant_smem(F k, std::atomic<size_t> &granted, size_t smem)
{
    if (smem <= granted.load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_grant_mutex);
    if (smem <= granted.load(std::memory_order_relaxed)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    granted.store(smem, std::memory_order_release);
    return cudaSuccess;
}

template <class R, int KER, int NT, bool PD = true>
static cudaError_t launch_t(const RolloutArgs &a, int grid, size_t smem, cudaStream_t s)
{
    auto k = rollout_kernel<R, KER, NT, PD>;
    // raise the kernel's dynamic shared-memory limit once per size increase (per process;
    // the library runs on one device per process)
    static std::atomic<size_t> granted{0};
    {
        const cudaError_t e = grant_smem(k, granted, smem);
        if (e != cudaSuccess) return e;
    }
    // binary32 multi-step launches that fit in one wave with several blocks per SM are paced
    RolloutArgs b = a;
    void *pace = nullptr;
    if (sizeof(R) == 4 && a.H > 1 && a.cap > kPaceMinCap && !a.pace_mask && pacing_requested()) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem) == cudaSuccess &&
            per_sm > 1 && grid > sms && grid <= per_sm * sms) {
            const int ids = kPaceSms;
            const size_t bytes = sizeof(unsigned) * ids + sizeof(int) * ids * kPaceSlots;
            if (lib_malloc_async(&pace, bytes, s) == cudaSuccess) {
                cudaError_t e = cudaMemsetAsync(pace, 0, bytes, s);
                if (e != cudaSuccess) {
                    cudaFreeAsync(pace, s);
                    return e;
                }
                b.pace_mask = static_cast<unsigned *>(pace);
                b.pace_prog = reinterpret_cast<int *>(b.pace_mask + ids);
                b.pace_sms = ids;
            } else {
                pace = nullptr;          // no pacing: a speed hint only
            }
        }
        cudaGetLastError();
    }
    k<<<grid, NT, smem, s>>>(b);
    cudaError_t e = cudaGetLastError();
    if (pace) {
        const cudaError_t e2 = cudaFreeAsync(pace, s);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

// Binary32 block size by field capacity: more warps where shared memory admits fewer blocks
// per SM (results do not depend on it).
template <int KER>
static cudaError_t launch_f32(const RolloutArgs &a, int grid, size_t smem, cudaStream_t s)
{
    if (a.cap > 3000) return launch_t<float, KER, 512>(a, grid, smem, s);
    if (a.cap > 1300) return launch_t<float, KER, 256>(a, grid, smem, s);
    if (a.cap >= kDiagPairMin) return launch_t<float, KER, 128, true>(a, grid, smem, s);
    return launch_t<float, KER, 128, false>(a, grid, smem, s);
}

long long rollout_rev_slots(int precision, int cap)
{
    return precision == VPM_FP64 ? 0 : rev_slots(cap);
}

long long rollout_scratch_slot(int cap, int kind, int row, int particle)
{
    return kind == 0 ? 2LL * fwd_index(particle) : rev_slot(row, particle, (cap + 31) & ~31);
}

// The library's own memory pool, one per device, for the stream-ordered scratch of its launches.
// Its release threshold is at its maximum, so scratch freed by one launch stays reserved for
// the next instead of going back to the device at every synchronisation; the device's default
// pool, which other code in the process uses, keeps its own settings.
static constexpr int kPoolDevices = 64;
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[kPoolDevices];

cudaMemPool_t lib_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kPoolDevices) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaGetLastError();
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    cudaMemPool_t pool = lib_pool();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

size_t lib_pool_idle_bytes()
{
    cudaMemPool_t pool = lib_pool();
    if (!pool) return 0;
    unsigned long long reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return reserved > used ? (size_t)(reserved - used) : 0;
}

// Runs launch(args) with the binary32 pair-sum scratch in place: the caller's, or one
// allocated on the stream for the launch's blocks and freed after it (stream-ordered, so
// launches on other streams get their own).
template <class F>
static cudaError_t with_rev_scratch(const RolloutArgs &a, int grid, cudaStream_t s, F launch)
{
    const long long slots = rev_slots(a.cap);
    if (slots == 0 || a.rev || a.H == 0) return launch(a);
    RolloutArgs b = a;
    void *buf = nullptr;
    cudaError_t e = lib_malloc_async(&buf, sizeof(float2) * (size_t)slots * (size_t)grid, s);
    if (e != cudaSuccess) return e;
    b.rev = static_cast<float2 *>(buf);
    b.rev_stride = slots;
    e = launch(b);
    const cudaError_t e2 = cudaFreeAsync(buf, s);
    return e != cudaSuccess ? e : e2;
}

size_t rollout_smem_bytes(int precision, int cap)
{
    return precision == VPM_FP64 ? (size_t)cap * (sizeof(Part64) + sizeof(double2))
                                 : (size_t)cap * (sizeof(float4) + sizeof(float2));
}

// Rollouts per launch up to which the binary64 path uses one cluster per rollout.
constexpr int kClusterRollouts = 9;

// Binary32 launches of few rollouts with large fields spread each rollout over a cluster of CTAs
// (the persistent cluster kernel of the uneven batch): with one CTA per rollout, K rollouts of
// fields that fit one CTA per SM use only K SMs. Measured over 50 steps (K x field): 64 x 6000
// 62.4 ms on one CTA, 36.9 ms on 2, 61.7 ms on 4; 32 x 8000 109.4, 59.1, 42.9 ms; 128 x 4000,
// 148 x 3000 and 512 x 2600 fastest on one CTA. Rule: the largest C in {4, 2} with K C <= SMs for
// fields that can exceed kClusterFieldMin particles (smaller fields: the plate warp's work,
// repeated on every CTA, is a larger share). Results are the same bits. VPM_ROLLOUT_CLUSTERS=0
// in the environment at launch keeps one CTA per rollout, and so does a launch made during stream
// capture for a launch shape no earlier launch has used (below).
constexpr int kClusterFieldMin = 2300;

// Resident clusters and the SM count by launch shape, remembered from launches made outside stream
// capture: a launch made while its stream is being captured must not query occupancy or raise a
// kernel's shared-memory limit (either invalidates the capture), so it uses clusters only for a
// shape an earlier launch has seen, and one block per rollout otherwise (the same bits).
struct ClusterShape { int nt, ctas; size_t smem; int clusters; };
static std::mutex g_cshape_mutex;
static ClusterShape g_cshapes[64];
static int g_ncshapes = 0;
static std::atomic<int> g_sms{0};

static int cached_clusters(int nt, int ctas, size_t smem, bool capturing)
{
    {
        std::lock_guard<std::mutex> lock(g_cshape_mutex);
        for (int i = 0; i < g_ncshapes; ++i)
            if (g_cshapes[i].nt == nt && g_cshapes[i].ctas == ctas && g_cshapes[i].smem == smem)
                return g_cshapes[i].clusters;
    }
    if (capturing) return 0;
    const int c = uneven_max_clusters(VPM_FP32, VPM_KERNEL_VATISTAS, nt, kDiagT, ctas, smem);
    std::lock_guard<std::mutex> lock(g_cshape_mutex);
    if (g_ncshapes < 64) g_cshapes[g_ncshapes++] = ClusterShape{nt, ctas, smem, c};
    return c;
}

static int rollout_cluster_size(const RolloutArgs &a, int grid, size_t smem, cudaStream_t s, bool &capturing)
{
    capturing = false;
    if (a.p.kernel != VPM_KERNEL_VATISTAS || a.H <= 1 || a.cap <= kClusterFieldMin || a.probe_fm ||
        a.probe_gs || a.probe_vel || a.probe_vt || a.pace_mask || a.order || a.counter)
        return 1;
    const char *env = getenv("VPM_ROLLOUT_CLUSTERS");
    if (env && env[0] == '0' && env[1] == 0) return 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    capturing = cs != cudaStreamCaptureStatusNone;
    int sms = g_sms.load(std::memory_order_acquire);
    if (!sms) {
        int dev = 0;
        if (capturing) return 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        g_sms.store(sms, std::memory_order_release);
    }
    const int nt = a.cap > 3000 ? 512 : 256;
    for (int c : {4, 2})
        if ((long long)grid * c <= sms && cached_clusters(nt, c, smem, capturing) >= 1) return c;
    return 1;
}

// `grid` rollouts (a.rid0 ...) as clusters of `ctas` CTAs claiming them from a counter of their own.
static cudaError_t launch_rollout_clusters(const RolloutArgs &a, int grid, int ctas, bool capturing,
                                          cudaStream_t s)
{
    const size_t smem = rollout_smem_bytes(VPM_FP32, a.cap);
    const int nt = a.cap > 3000 ? 512 : 256;
    const int clusters = std::min(grid, cached_clusters(nt, ctas, smem, capturing));
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    void *cnt = nullptr;
    cudaError_t e = lib_malloc_async(&cnt, sizeof(int), s);
    if (e != cudaSuccess) return e;
    RolloutArgs b = a;
    b.counter = static_cast<int *>(cnt);
    b.order = nullptr;
    b.n_items = grid;
    e = cudaMemsetAsync(cnt, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_uneven_cluster(b, clusters, nt, kDiagT, ctas, s);
    const cudaError_t e2 = cudaFreeAsync(cnt, s);
    return e != cudaSuccess ? e : e2;
}
template <int KER>
static cudaError_t launch_cluster_t(const RolloutArgs &a, int grid, size_t smem, cudaStream_t s);

cudaError_t launch_rollout(int precision, const RolloutArgs &a, int grid, cudaStream_t s)
{
    const size_t smem = rollout_smem_bytes(precision, a.cap);
    const int ker = a.p.kernel;
    if (precision == VPM_FP64) {
        // a few multi-step rollouts without single-step probes: one cluster of SMs per rollout
        if (grid <= kClusterRollouts && a.H > 1 && !a.probe_fm && !a.probe_gs && !a.probe_vel && !a.probe_vt) {
            if (ker == VPM_KERNEL_GAUSSIAN) return launch_cluster_t<VPM_KERNEL_GAUSSIAN>(a, grid, smem, s);
            if (ker == VPM_KERNEL_SINGULAR) return launch_cluster_t<VPM_KERNEL_SINGULAR>(a, grid, smem, s);
            return launch_cluster_t<VPM_KERNEL_VATISTAS>(a, grid, smem, s);
        }
        if (ker == VPM_KERNEL_GAUSSIAN) return launch_t<double, VPM_KERNEL_GAUSSIAN, 128>(a, grid, smem, s);
        if (ker == VPM_KERNEL_SINGULAR) return launch_t<double, VPM_KERNEL_SINGULAR, 128>(a, grid, smem, s);
        return launch_t<double, VPM_KERNEL_VATISTAS, 128>(a, grid, smem, s);
    }
    bool capturing = false;
    const int ctas = rollout_cluster_size(a, grid, smem, s, capturing);
    if (ctas > 1)
        return with_rev_scratch(a, grid, s, [&](const RolloutArgs &b) {
            return launch_rollout_clusters(b, grid, ctas, capturing, s);
        });
    return with_rev_scratch(a, grid, s, [&](const RolloutArgs &b) {
        if (ker == VPM_KERNEL_GAUSSIAN) return launch_f32<VPM_KERNEL_GAUSSIAN>(b, grid, smem, s);
        if (ker == VPM_KERNEL_SINGULAR) return launch_f32<VPM_KERNEL_SINGULAR>(b, grid, smem, s);
        return launch_f32<VPM_KERNEL_VATISTAS>(b, grid, smem, s);
    });
}

template <class R, int KER, int NT, int DT = kDiagT, bool PD = true>
static cudaError_t launch_u(const RolloutArgs &a, int grid, size_t smem, cudaStream_t s)
{
    auto k = uneven_kernel<R, KER, NT, DT, PD>;
    static std::atomic<size_t> granted{0};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusNone) {         // under capture the batch raised it before
        const cudaError_t e = grant_smem(k, granted, smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

// Block size nt and diagonal-unit targets per lane dt (1, 2 or 4; other than kDiagT only for the
// Vatistas kernel of Eq. 5, the workloads' kernel) of the binary32 persistent launch.
template <class R, int KER>
static cudaError_t launch_u_nt(const RolloutArgs &a, int grid, int nt, int dt, size_t smem, cudaStream_t s)
{
    if (KER == VPM_KERNEL_VATISTAS && dt == 1) {
        if (nt == 512) return launch_u<R, KER, 512, 1>(a, grid, smem, s);
        if (nt == 256) return launch_u<R, KER, 256, 1>(a, grid, smem, s);
        if (a.cap < kDiagPairMin) return launch_u<R, KER, 128, 1, false>(a, grid, smem, s);
        return launch_u<R, KER, 128, 1>(a, grid, smem, s);
    }
    if (KER == VPM_KERNEL_VATISTAS && dt == 4) {
        if (nt == 512) return launch_u<R, KER, 512, 4>(a, grid, smem, s);
        if (nt == 256) return launch_u<R, KER, 256, 4>(a, grid, smem, s);
        if (a.cap < kDiagPairMin) return launch_u<R, KER, 128, 4, false>(a, grid, smem, s);
        return launch_u<R, KER, 128, 4>(a, grid, smem, s);
    }
    if (nt == 512) return launch_u<R, KER, 512>(a, grid, smem, s);
    if (nt == 256) return launch_u<R, KER, 256>(a, grid, smem, s);
    if (a.cap < kDiagPairMin) return launch_u<R, KER, 128, kDiagT, false>(a, grid, smem, s);
    return launch_u<R, KER, 128>(a, grid, smem, s);
}

cudaError_t launch_uneven(int precision, const RolloutArgs &a, int grid, int nt, int dt, cudaStream_t s)
{
    const size_t smem = rollout_smem_bytes(precision, a.cap);
    const int ker = a.p.kernel;
    if (precision == VPM_FP64) {
        if (ker == VPM_KERNEL_GAUSSIAN) return launch_u<double, VPM_KERNEL_GAUSSIAN, 128>(a, grid, smem, s);
        if (ker == VPM_KERNEL_SINGULAR) return launch_u<double, VPM_KERNEL_SINGULAR, 128>(a, grid, smem, s);
        return launch_u<double, VPM_KERNEL_VATISTAS, 128>(a, grid, smem, s);
    }
    return with_rev_scratch(a, grid, s, [&](const RolloutArgs &b) {
        if (ker == VPM_KERNEL_GAUSSIAN) return launch_u_nt<float, VPM_KERNEL_GAUSSIAN>(b, grid, nt, dt, smem, s);
        if (ker == VPM_KERNEL_SINGULAR) return launch_u_nt<float, VPM_KERNEL_SINGULAR>(b, grid, nt, dt, smem, s);
        return launch_u_nt<float, VPM_KERNEL_VATISTAS>(b, grid, nt, dt, smem, s);
    });
}

// Sets the kernel's dynamic shared-memory limit to at least smem and returns the resident
// blocks per SM.
template <class F>
static int occupancy_of(F k, int nt, size_t smem)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nt, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

int uneven_blocks_per_sm(int precision, int kernel, int nt, int dt, size_t smem)
{
    if (precision == VPM_FP64) {
        if (kernel == VPM_KERNEL_GAUSSIAN) return occupancy_of(uneven_kernel<double, VPM_KERNEL_GAUSSIAN, 128>, 128, smem);
        if (kernel == VPM_KERNEL_SINGULAR) return occupancy_of(uneven_kernel<double, VPM_KERNEL_SINGULAR, 128>, 128, smem);
        return occupancy_of(uneven_kernel<double, VPM_KERNEL_VATISTAS, 128>, 128, smem);
    }
    if (kernel == VPM_KERNEL_VATISTAS && (dt == 1 || dt == 4)) {
        if (dt == 1) {
            if (nt == 512) return occupancy_of(uneven_kernel<float, VPM_KERNEL_VATISTAS, 512, 1>, 512, smem);
            if (nt == 256) return occupancy_of(uneven_kernel<float, VPM_KERNEL_VATISTAS, 256, 1>, 256, smem);
            return occupancy_of(uneven_kernel<float, VPM_KERNEL_VATISTAS, 128, 1>, 128, smem);
        }
        if (nt == 512) return occupancy_of(uneven_kernel<float, VPM_KERNEL_VATISTAS, 512, 4>, 512, smem);
        if (nt == 256) return occupancy_of(uneven_kernel<float, VPM_KERNEL_VATISTAS, 256, 4>, 256, smem);
        return occupancy_of(uneven_kernel<float, VPM_KERNEL_VATISTAS, 128, 4>, 128, smem);
    }
#define VPM_OCC(KER)                                                                         \
    if (nt == 512) return occupancy_of(uneven_kernel<float, KER, 512>, 512, smem);           \
    if (nt == 256) return occupancy_of(uneven_kernel<float, KER, 256>, 256, smem);           \
    return occupancy_of(uneven_kernel<float, KER, 128>, 128, smem);
    if (kernel == VPM_KERNEL_GAUSSIAN) { VPM_OCC(VPM_KERNEL_GAUSSIAN) }
    if (kernel == VPM_KERNEL_SINGULAR) { VPM_OCC(VPM_KERNEL_SINGULAR) }
    VPM_OCC(VPM_KERNEL_VATISTAS)
#undef VPM_OCC
}

// Cluster launches of the binary32 persistent kernel (Vatistas kernel of Eq. 5, the workloads'
// kernel): `clusters` clusters of `ctas` CTAs of nt threads, diagonal units of 32 dt targets.
template <int NT, int DT>
static cudaLaunchConfig_t cluster_cfg_u(int clusters, int ctas, size_t smem, cudaStream_t s,
                                        cudaLaunchAttribute &at)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * ctas);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = ctas; at.val.clusterDim.y = 1; at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cfg;
}

template <int NT, int DT>
static std::atomic<size_t> &granted_uc()
{
    static std::atomic<size_t> g{0};
    return g;
}

template <int NT, int DT>
static int clusters_uc(int ctas, size_t smem)
{
    auto k = uneven_cluster_kernel<VPM_KERNEL_VATISTAS, NT, DT>;
    if (grant_smem(k, granted_uc<NT, DT>(), smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute at;
    cudaLaunchConfig_t cfg = cluster_cfg_u<NT, DT>(1, ctas, smem, nullptr, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <int NT, int DT>
static cudaError_t launch_uc(const RolloutArgs &a, int clusters, int ctas, size_t smem, cudaStream_t s)
{
    auto k = uneven_cluster_kernel<VPM_KERNEL_VATISTAS, NT, DT>;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusNone) {         // under capture the batch raised it before
        const cudaError_t e = grant_smem(k, granted_uc<NT, DT>(), smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchAttribute at;
    const cudaLaunchConfig_t cfg = cluster_cfg_u<NT, DT>(clusters, ctas, smem, s, at);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int uneven_max_clusters(int precision, int kernel, int nt, int dt, int ctas, size_t smem)
{
    if (precision != VPM_FP32 || kernel != VPM_KERNEL_VATISTAS || (ctas != 2 && ctas != 4)) return 0;
#define VPM_UC(NT_)                                                   \
    if (nt == NT_) {                                                  \
        if (dt == 1) return clusters_uc<NT_, 1>(ctas, smem);          \
        if (dt == 4) return clusters_uc<NT_, 4>(ctas, smem);          \
        return clusters_uc<NT_, 2>(ctas, smem);                       \
    }
    VPM_UC(512)
    VPM_UC(256)
    VPM_UC(128)
#undef VPM_UC
    return 0;
}

cudaError_t launch_uneven_cluster(const RolloutArgs &a, int clusters, int nt, int dt, int ctas,
                                  cudaStream_t s)
{
    if (a.p.kernel != VPM_KERNEL_VATISTAS || (ctas != 2 && ctas != 4) || clusters < 1 ||
        (rev_slots(a.cap) > 0 && (!a.rev || a.rev_stride < rev_slots(a.cap))))
        return cudaErrorInvalidValue;
    const size_t smem = rollout_smem_bytes(VPM_FP32, a.cap);
#define VPM_UC(NT_)                                                         \
    if (nt == NT_) {                                                        \
        if (dt == 1) return launch_uc<NT_, 1>(a, clusters, ctas, smem, s);  \
        if (dt == 4) return launch_uc<NT_, 4>(a, clusters, ctas, smem, s);  \
        return launch_uc<NT_, 2>(a, clusters, ctas, smem, s);               \
    }
    VPM_UC(512)
    VPM_UC(256)
    VPM_UC(128)
#undef VPM_UC
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ one binary64 rollout per cluster

// A few binary64 rollouts (a single simulation, such as the fixed plate in a stream) spread over a thread-block
// cluster: every CTA holds the whole field; the plate-point sums and the convection targets are
// split across the CTAs, each CTA broadcasts its results (plate velocities, advected records) to
// every CTA's shared memory through distributed shared memory, and hardware cluster barriers
// separate the phases. The small serial plate work (geometry, solve, loads, glider, shedding,
// termination, merging) runs redundantly on every CTA from identical data. Every target's sum is
// formed in the same order as on the one-block path, so the results are the same bits.
template <int KER>
__global__ void __launch_bounds__(kThreads) cluster_rollout_kernel(const RolloutArgs a)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int rid = (int)(blockIdx.x / C) + a.rid0;
    extern __shared__ __align__(16) unsigned char smem[];
    Part64 *part = reinterpret_cast<Part64 *>(smem);
    double2 *vel = reinterpret_cast<double2 *>(smem + sizeof(Part64) * (size_t)a.cap);
    __shared__ Work w;
    const DevParams &p = a.p;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = (int)(blockDim.x >> 5);
    load_state<double>(a, w, part, rid);
    int n = w.n;
    cl.sync();
    for (int k = 0; k < a.H; ++k) {
        double u = a.controls ? (double)a.controls[(size_t)rid * a.ctrl_stride + a.step0 + k] : a.u_const;
        if (a.pol_gains && warp == 0) {
            const size_t j = (size_t)a.pol_offset + k;
            double fb = (double)a.pol_ubar[j];
            for (int c = 0; c < 7; ++c) fb -= a.pol_gains[j * 7 + c] * (w.xg[c] - a.pol_xbar[j * 7 + c]);
            u = (a.controls ? u : 0.0) + fb;
        }
        if (warp == 0) plate_geometry(p, w);
        __syncthreads();
        // plate-point sums (Eq. 12): target t on CTA t mod C, written into every CTA
        const int M = p.n_c + p.n_b;
        for (int t = rank + C * warp; t < M; t += C * nwarps) {
            double tx, tz;
            plate_point(p, w.geo, t, tx, tz);
            double su = 0.0, sw = 0.0;
            for (int j = lane; j < n; j += 32) {
                const Part64 sj = part[j];
                const double dx = tx - sj.x, dz = tz - sj.z;
                const double g = sj.g * PairF64<KER>::q(fma(dx, dx, dz * dz), p.rc4, p.inv_rc2);
                su = fma(-dz, g, su);
                sw = fma(dx, g, sw);
            }
            for (int o = 16; o > 0; o >>= 1) {
                su += __shfl_xor_sync(0xffffffffu, su, o);
                sw += __shfl_xor_sync(0xffffffffu, sw, o);
            }
            if (lane < C) {
                double *rv = cl.map_shared_rank(&w.vt[0], lane);
                rv[2 * t] = su * kInv2Pi;
                rv[2 * t + 1] = sw * kInv2Pi;
            }
        }
        // Kelvin sum (Eq. 7), the same partition as the one-block path, on every CTA
        double gsum = 0.0;
        for (int j = tid; j < n; j += (int)blockDim.x) gsum += part[j].g;
        for (int o = 16; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
        if (lane == 0) w.red[warp] = gsum;
        cl.sync();
        if (warp == 0) {
            const int m = plate_solve<double>(p, w, part, n, u, nwarps);
            if (lane == 0) w.n = m;
        }
        __syncthreads();
        const int n1 = w.n;
        // convection of this CTA's slice of targets (Eq. 16), one warp per target in the
        // one-block order (convect_target_f64)
        const int per = (n1 + C - 1) / C, lo = min(n1, rank * per), hi = min(n1, lo + per);
        const int slot0 = warp + nwarps * lane, slot_step = nwarps * 32;
        for (int i = lo + warp; i < hi; i += nwarps) {
            const Part64 pi = part[i];
            const double2 v = convect_target_f64<KER>(p, w, part, n1, pi.x, pi.z);
            if (lane == 0) vel[i] = v;
        }
        __syncthreads();                             // vel of the slice is complete in this CTA
        cl.sync();                                   // every CTA is done reading the positions
        bool bad = false;
        for (int i = lo + slot0; i < hi; i += slot_step) {
            Part64 q = part[i];
            const double2 v = vel[i];
            bad |= !(isfinite(v.x) && isfinite(v.y));
            q.x += p.dt * v.x;
            q.z += p.dt * v.y;
            q.g *= p.decay;
            for (int r = 0; r < C; ++r) cl.map_shared_rank(part, r)[i] = q;
        }
        if (bad) atomicOr(&w.flag, (int)kStNonFinite);
        cl.sync();                                   // the advected field is complete everywhere
        int nn = n1;
        if (w.ndist == 2) nn = terminate_pair<double>(p, w, part, nn);
        n = merge_oldest<double>(p, part, nn, w.ndist);
        if (rank == 0 && a.traj && tid < 7) a.traj[((size_t)rid * a.H + k) * 7 + tid] = w.xg[tid];
    }
    if (tid == 0) {
        w.n = n;
        if (rank != 0 && w.flag) atomicOr(cl.map_shared_rank(&w.flag, 0), w.flag);
    }
    cl.sync();
    if (rank == 0) {
        if (a.out_part) store_state<double>(a, w, part, rid);
        finish<double>(a, w, part, rid);
    }
}

template <int KER>
static cudaError_t launch_cluster_t(const RolloutArgs &a, int grid, size_t smem, cudaStream_t s)
{
    auto k = cluster_rollout_kernel<KER>;
    static std::atomic<size_t> granted{0};
    static std::atomic<int> csize_cached{0};
    {
        const cudaError_t e = grant_smem(k, granted, smem);
        if (e != cudaSuccess) return e;
    }
    int csize = csize_cached.load(std::memory_order_acquire);
    if (!csize) {                                    // 16 CTAs where the part allows, else 8
        std::lock_guard<std::mutex> lock(g_grant_mutex);
        csize = 8;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3(16);
            q.blockDim = dim3(kThreads);
            q.dynamicSmemBytes = smem;
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = 16; at.val.clusterDim.y = 1; at.val.clusterDim.z = 1;
            q.attrs = &at;
            q.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, k, &q) == cudaSuccess && clusters > 0) csize = 16;
        }
        cudaGetLastError();
        csize_cached.store(csize, std::memory_order_release);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid * csize);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = csize; attr.val.clusterDim.y = 1; attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ disturbance injection

template <class R>
__global__ void __launch_bounds__(kThreads) inject_pair_kernel(typename Store<R>::P *part, int *d_n,
                                                              int cap, double x1, double z1,
                                                              double g1, double x2, double z2,
                                                              double g2)
{
    using P = typename Store<R>::P;
    const int n = d_n[0];
    if (kDebugBounds && n + 2 > cap) return;         // the host checked the capacity
    // move records up by two, top chunk first (each chunk's targets are read before written)
    for (int top = n; top > 0; top -= (int)blockDim.x) {
        const int i = top - 1 - (int)threadIdx.x;
        P tmp;
        if (i >= 0) tmp = part[i];
        __syncthreads();
        if (i >= 0) part[i + 2] = tmp;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[0] = Store<R>::make(x1, z1, g1);
        part[1] = Store<R>::make(x2, z2, g2);
        d_n[0] = n + 2;
        d_n[1] = 2;
    }
}

cudaError_t launch_inject_pair(int precision, void *d_part, int *d_n, int cap, const double *pair,
                               cudaStream_t s)
{
    if (precision == VPM_FP64)
        inject_pair_kernel<double><<<1, kThreads, 0, s>>>(static_cast<Part64 *>(d_part), d_n, cap,
                                                          pair[0], pair[1], pair[2], pair[3], pair[4], pair[5]);
    else
        inject_pair_kernel<float><<<1, kThreads, 0, s>>>(static_cast<float4 *>(d_part), d_n, cap,
                                                         pair[0], pair[1], pair[2], pair[3], pair[4], pair[5]);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pair-loop throughput probe

template <int T>
__global__ void __launch_bounds__(kThreads, VPM_MIN_BLOCKS) pair_probe_kernel(const float4 *src,
                                                                            float2 *out, int n,
                                                                            int reps, float rc4)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *part = reinterpret_cast<float4 *>(smem);
    float2 *vel = reinterpret_cast<float2 *>(smem + sizeof(float4) * (size_t)n);
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) part[i] = src[i];
    __syncthreads();
    DevParams p = {};
    p.rc4 = rc4;
    const int warp = threadIdx.x >> 5, nwarps = (int)blockDim.x >> 5;
    for (int r = 0; r < reps; ++r)
        for (int base = 32 * T * warp; base < n; base += 32 * T * nwarps)
            old_pairs_chunk<VPM_KERNEL_VATISTAS, T>(p, part, vel, 0, n, base, n);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) out[(size_t)blockIdx.x * n + i] = vel[i];
}

// The rollout kernel's binary32 pair phase as it runs (rows with one evaluation per pair,
// diagonal groups, claims from a shared counter, then every particle's partial sums combined),
// `reps` times over the same n records.
__global__ void __launch_bounds__(kThreads, VPM_MIN_BLOCKS) pair_probe_sym_kernel(const float4 *src,
                                                                              float2 *out,
                                                                              float2 *scratch,
                                                                              long long stride,
                                                                              int n, int reps,
                                                                              float rc4)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *part = reinterpret_cast<float4 *>(smem);
    float2 *vel = reinterpret_cast<float2 *>(smem + sizeof(float4) * (size_t)n);
    __shared__ Work w;
    for (int i = threadIdx.x; i < n; i += (int)blockDim.x) part[i] = src[i];
    if (threadIdx.x == 0) w.chunk_next = 0;
    __syncthreads();
    DevParams p = {};
    p.rc4 = rc4;
    float2 *scr = scratch + (size_t)blockIdx.x * stride;
    const PairPlan pp = pair_plan(n);
    const int cap32 = (n + 31) & ~31;
    int claim_base = 0;
    for (int r = 0; r < reps; ++r) {
        old_pairs_f32<VPM_KERNEL_VATISTAS>(p, w, part, vel, scr, cap32, n, pp, claim_base);
        claim_base += pp.nunits + (int)(blockDim.x >> 5);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += (int)blockDim.x) {
            const float2 v = old_sum(vel, scr, cap32, pp.rows_off, i);
            if (r == reps - 1) out[(size_t)blockIdx.x * n + i] = v;
        }
        __syncthreads();
    }
}

cudaError_t launch_pair_probe_sym(int grid, int n, int reps, double r_core, const float4 *d_src,
                                  float2 *d_out, float2 *d_scratch, cudaStream_t s)
{
    const size_t smem = (size_t)n * (sizeof(float4) + sizeof(float2));
    const float rc4 = (float)(r_core * r_core * r_core * r_core);
    cudaError_t e = cudaFuncSetAttribute(pair_probe_sym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    pair_probe_sym_kernel<<<grid, kThreads, smem, s>>>(d_src, d_out, d_scratch, rev_slots(n), n, reps, rc4);
    return cudaGetLastError();
}

cudaError_t launch_pair_probe(int t, int grid, int n, int reps, double r_core, const float4 *d_src,
                              float2 *d_out, cudaStream_t s)
{
    const size_t smem = (size_t)n * (sizeof(float4) + sizeof(float2));
    const float rc4 = (float)(r_core * r_core * r_core * r_core);
    auto k = t == 4 ? pair_probe_kernel<4> : (t == 2 ? pair_probe_kernel<2> : pair_probe_kernel<1>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kThreads, smem, s>>>(d_src, d_out, n, reps, rc4);
    return cudaGetLastError();
}

}  // namespace vpm
