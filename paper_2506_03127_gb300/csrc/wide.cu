// The MACGIC-iQUAPI path update with keys of up to 128 bits: M up to 8
// system states and windows of up to 16 points (the production models of
// Sec. 4.3 need M = 8 at Delta k_max = 12, 72 bits with two 3-bit states per
// point).  A stored key holds one byte per window position (position 0 =
// newest point in the lowest byte): the forward state in the low nibble,
// the backward state in the high one, in two 64-bit words (lo: positions
// 0..7, hi: 8..15).  The order of these keys, as 128-bit numbers, compares
// the oldest position first and the backward state before the forward one:
// the order of the packed keys of the narrow engines, so the tie rule of
// the pre-merge (reading R4) is the same.
//
// One step (Sec. 3.1, Schemes merging and propagation), pre-merging order:
//   k_w_insert  group every stored path by its P' positions (a 64-bit group
//               key of 6 bits per position) in an open-addressing table:
//               FP64 sums, largest weight (Sec. 3.1 "Pre-merging");
//   k_w_tie     members within the tie window of the largest weight compete
//               on a 64-bit tie key (the positions outside P', in key order);
//   (k_w_tie<true>: the winner becomes the group's representative)
//   k_w_expand  the M^2 children of each group (Eqs. SysP, inf_fun), one at
//               a time: one lane per group, or sub_n lanes sharing a group,
//               each forming every sub_n-th child; the history part H of the
//               influence exponent from per-position tables; filtered
//               (|amp| >= theta, Sec. 2.1) and appended in output ranges
//               reserved once per block and round;
//   k_w_rho     rho(t) from the appended children by newest point (Eq.
//               quapi_red_rho), per-block sums;
//   k_w_finalize the step's rho, counts and state.
// While the window fills every stored path is its own group (reading R3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr int kWMaxM = 8, kWMaxDk = 16, kWMaxMM = 64;
constexpr int kWThreads = 256;
constexpr int kWProbe = 64;
constexpr int kWMaxTabDelta = 16;   // distinct coupling differences up to which a group tabulates its factors
constexpr unsigned long long kWEmpty = ~0ull;
constexpr unsigned kWErrPaths = 1u, kWErrGroups = 2u, kWErrProbe = 4u;

struct WState {
    unsigned long long t, n_cur;       // stored set Omega(t) and its size
    unsigned long long n_groups;       // groups of the running step
    unsigned long long n_out;          // children appended by the running step
    unsigned int err;                  // sticky error bits
    unsigned int pad;
};

struct WRec { long long t, groups, extended, kept, inter; };

// a merge-table slot: group key, largest weight (FP64 bits) and the FP64
// sum in one 32-byte sector
struct __align__(32) WSlot {
    unsigned long long gk, wm;
    double sre, sim;
};

struct WParams {
    int M, dkmax, c64, rho_hist;
    long long max_paths, max_groups;
    unsigned long long tcap_mask;
    int npp, nco;                      // positions of P' and of its complement (ascending)
    int pp[kWMaxDk], co[kWMaxDk];
    double theta2, tie_rel;
    float theta2f;
    double q[kWMaxM];
    int ndelta;                        // distinct nonzero q_a - q_b (tabulated per group when <= kWMaxTabDelta)
    double delta[kWMaxMM];
    signed char dsel[kWMaxMM];         // child c -> its difference (-1: q_a = q_b)
    unsigned long long *klo[2], *khi[2];
    void *amps[2];
    unsigned int *slot_of, *groups, *trep;
    WSlot *slots;
    unsigned long long *ttie;
    const double2 *lut;                // [dkmax][dkmax - 1][256] FP64 history tables
    const float2 *lutf, *lutlo;        // FP32 hi part and residual
    const double2 *w;                  // [M*M child][M*M parent newest]
    const float4 *wf;                  // FP32 hi/lo pairs of w
    double2 *rho_part;                 // [blocks][M*M]
    double2 *rho_ring;                 // [rho_hist][M*M]
    WRec *stats;                       // [rho_hist]
    WState *st;
};

__device__ __forceinline__ unsigned key_byte(unsigned long long lo, unsigned long long hi, int j) {
    return (unsigned)((j < 8 ? lo >> (8 * j) : hi >> (8 * (j - 8))) & 0xffull);
}
// 6-bit code of a position (forward | backward << 3), positions in ascending
// order at ascending bits: equal on P' <=> equal group keys; on the
// complement the order of the full keys
__device__ __forceinline__ unsigned long long pack6(unsigned long long lo, unsigned long long hi, const int *pos,
                                                    int n) {
    unsigned long long k = 0;
    for (int i = 0; i < n; ++i) {
        const unsigned v = key_byte(lo, hi, pos[i]);
        k |= (unsigned long long)((v & 7u) | (((v >> 4) & 7u) << 3)) << (6 * i);
    }
    return k;
}
__device__ __forceinline__ unsigned long long wmix(unsigned long long x) {
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}
__device__ __forceinline__ double weight_of(const WParams &P, const void *amps, unsigned long long i) {
    if (P.c64) {
        const float2 a = static_cast<const float2 *>(amps)[i];
        return (double)(a.x * a.x + a.y * a.y);
    }
    const double2 a = static_cast<const double2 *>(amps)[i];
    return a.x * a.x + a.y * a.y;
}
__device__ __forceinline__ double2 amp_of(const WParams &P, const void *amps, unsigned long long i) {
    if (P.c64) {
        const float2 a = static_cast<const float2 *>(amps)[i];
        return make_double2(a.x, a.y);
    }
    return static_cast<const double2 *>(amps)[i];
}

// pre-merge, pass 1: claim or find the group's slot, add the amplitude,
// raise the largest weight
__global__ void k_w_insert(WParams P) {
    WState *st = P.st;
    if (st->err) return;
    const int in = (int)(st->t & 1);
    const unsigned long long n = st->n_cur;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long lo = P.klo[in][i], hi = P.khi[in][i];
        const unsigned long long gk = pack6(lo, hi, P.pp, P.npp);
        unsigned long long h = wmix(gk) & P.tcap_mask;
        int probe = 0;
        for (; probe < kWProbe; ++probe, h = (h + 1) & P.tcap_mask) {
            unsigned long long cur = P.slots[h].gk;
            if (cur == kWEmpty) {
                cur = atomicCAS(&P.slots[h].gk, kWEmpty, gk);
                if (cur == kWEmpty) {   // claimed: a new group
                    const unsigned long long g = atomicAdd(&st->n_groups, 1ull);
                    if ((long long)g < P.max_groups) P.groups[g] = (unsigned)h;
                    else atomicOr(&st->err, kWErrGroups);
                    break;
                }
            }
            if (cur == gk) break;
        }
        if (probe == kWProbe) {
            atomicOr(&st->err, kWErrProbe);
            return;
        }
        const double2 a = amp_of(P, P.amps[in], i);
        atomicAdd(&P.slots[h].sre, a.x);
        atomicAdd(&P.slots[h].sim, a.y);
        atomicMax(&P.slots[h].wm, (unsigned long long)__double_as_longlong(weight_of(P, P.amps[in], i)));
        P.slot_of[i] = (unsigned)h;
    }
}

// pre-merge, pass 2: members within the tie window compete on the tie key
// (pass 3: the winner, unique in its group, becomes the representative)
template <bool REP>
__global__ void k_w_tie(WParams P) {
    WState *st = P.st;
    if (st->err) return;
    const int in = (int)(st->t & 1);
    const unsigned long long n = st->n_cur;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned h = P.slot_of[i];
        const double wm = __longlong_as_double((long long)P.slots[h].wm);
        if (weight_of(P, P.amps[in], i) < (1.0 - P.tie_rel) * wm) continue;
        const unsigned long long tk = pack6(P.klo[in][i], P.khi[in][i], P.co, P.nco);
        if (!REP) atomicMin(&P.ttie[h], tk);
        else if (tk == P.ttie[h]) P.trep[h] = (unsigned)i;
    }
}

// children of one group, appended in warp-aggregated blocks; thread-uniform
// loops (every lane of a warp runs every child, valid or not)
template <bool C64, bool TAB>
__global__ void __launch_bounds__(kWThreads) k_w_expand(WParams P, int merge, int sub_n) {
    // sub_n consecutive lanes share a group (a power of two dividing 32), lane
    // s taking its children c = s, s + sub_n, ...; each lane forms the
    // group's history sum itself.  TAB: the influence factors exp(-delta H)
    // of the group's distinct coupling differences, computed once per lane
    // (the same arithmetic as per child), in shared memory [delta][thread]
    using CT = typename std::conditional<C64, float2, double2>::type;
    extern __shared__ __align__(16) unsigned char s_wtab[];
    CT *sE = reinterpret_cast<CT *>(s_wtab);
    __shared__ unsigned s_wc[kWThreads / 32];
    __shared__ unsigned long long s_base;
    WState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    const int in = (int)(t & 1), outp = (int)(tn & 1);
    const unsigned long long ng = merge ? st->n_groups : st->n_cur;
    const int M = P.M, MM = M * M;
    const int n_act = (int)min(tn, (unsigned long long)P.dkmax);
    const int L_child = (int)min(tn + 1, (unsigned long long)P.dkmax);
    const int nb = P.dkmax - 1;                       // history bytes of a key
    const unsigned lane = threadIdx.x & 31u;
    const size_t row = (size_t)(n_act - 1) * nb * 256;
    const int sub = (int)(threadIdx.x & (unsigned)(sub_n - 1));
    for (unsigned long long base = blockIdx.x * (unsigned long long)blockDim.x; base < ng * sub_n;
         base += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long g = (base + threadIdx.x) / (unsigned)sub_n;
        const bool valid = g < ng;
        unsigned long long lo = 0, hi = 0;
        double2 S = make_double2(0.0, 0.0);
        unsigned h = 0;
        if (valid) {
            unsigned long long r = g;
            if (merge) {
                h = P.groups[g];
                r = P.trep[h];
                S = make_double2(P.slots[h].sre, P.slots[h].sim);
            } else {
                S = amp_of(P, P.amps[in], r);
            }
            lo = P.klo[in][r];
            hi = P.khi[in][r];
        }
        __syncwarp();   // every lane of the group has read the slot
        if (valid && merge && sub == 0) {   // read by this group only: reset it for the next step
            WSlot fresh;
            fresh.gk = kWEmpty;
            fresh.wm = 0ull;
            fresh.sre = fresh.sim = 0.0;
            P.slots[h] = fresh;
            P.ttie[h] = kWEmpty;
        }
        const int par = (int)(lo & 0xffull);
        const int parc = (par & 15) * M + (par >> 4);   // (forward, backward) of the newest point
        // history part H of the influence exponent: FP64, or FP32 with the
        // rounding of every addition kept (Kahan) from the hi/lo tables
        double Hx = 0.0, Hy = 0.0;
        float hx = 0.f, hy = 0.f, cx = 0.f, cy = 0.f;
        for (int j = 0; j < nb; ++j) {
            const unsigned v = key_byte(lo, hi, j);
            if constexpr (C64) {
                const float2 a = P.lutf[row + (size_t)j * 256 + v], b = P.lutlo[row + (size_t)j * 256 + v];
                float yx = (a.x - cx), tx = hx + yx;
                cx = (tx - hx) - yx;
                hx = tx;
                yx = (b.x - cx);
                tx = hx + yx;
                cx = (tx - hx) - yx;
                hx = tx;
                float yy = (a.y - cy), ty = hy + yy;
                cy = (ty - hy) - yy;
                hy = ty;
                yy = (b.y - cy);
                ty = hy + yy;
                cy = (ty - hy) - yy;
                hy = ty;
            } else {
                const double2 e = P.lut[row + (size_t)j * 256 + v];
                Hx += e.x;
                Hy += e.y;
            }
        }
        if constexpr (TAB) {
            for (int d = 0; d < P.ndelta; ++d) {
                if constexpr (C64) {
                    const float dqf = (float)P.delta[d];
                    const float zr = -dqf * hx, zi = -dqf * hy;
                    float sn, cs;
                    sincosf(zi, &sn, &cs);
                    const float m = expf(zr);
                    sE[d * kWThreads + threadIdx.x] = make_float2(m * cs, m * sn);
                } else {
                    const double zr = -P.delta[d] * Hx, zi = -P.delta[d] * Hy;
                    double sn, cs;
                    sincos(zi, &sn, &cs);
                    const double m = exp(zr);
                    sE[d * kWThreads + threadIdx.x] = make_double2(m * cs, m * sn);
                }
            }
        }
        // child key: the parent shifted up one position, the new point in
        // the lowest byte, cut to L_child positions
        unsigned long long chi = (hi << 8) | (lo >> 56), clo = lo << 8;
        if (8 * L_child <= 64) {
            chi = 0;
            if (8 * L_child < 64) clo &= (1ull << (8 * L_child)) - 1ull;
        } else if (8 * L_child < 128) {
            chi &= (1ull << (8 * L_child - 64)) - 1ull;
        }
        // child c of the group: its amplitude and whether it survives the filter
        auto child_of = [&](int c, double2 &child) -> bool {
            const int a = c / M, b = c % M;
            const double dq = P.q[a] - P.q[b];
            if constexpr (C64) {
                float fx, fy;
                if constexpr (TAB) {
                    const int d = P.dsel[c];
                    const float2 e = d < 0 ? make_float2(1.f, 0.f) : sE[d * kWThreads + threadIdx.x];
                    fx = e.x;
                    fy = e.y;
                } else {
                    const float dqf = (float)dq;
                    const float zr = -dqf * hx, zi = -dqf * hy;
                    float sn, cs;
                    sincosf(zi, &sn, &cs);
                    const float m = expf(zr);
                    fx = m * cs;
                    fy = m * sn;
                }
                const float4 wv = P.wf[(size_t)c * MM + parc];
                const float Sx = (float)S.x, Sy = (float)S.y;
                // S (W_hi + W_lo) f
                const float px = fmaf(Sx, wv.x, -Sy * wv.y) + fmaf(Sx, wv.z, -Sy * wv.w);
                const float py = fmaf(Sx, wv.y, Sy * wv.x) + fmaf(Sx, wv.w, Sy * wv.z);
                const float ox = px * fx - py * fy, oy = px * fy + py * fx;
                child = make_double2(ox, oy);
                return ox * ox + oy * oy >= P.theta2f;
            } else {
                double fx, fy;
                if constexpr (TAB) {
                    const int d = P.dsel[c];
                    const double2 e = d < 0 ? make_double2(1.0, 0.0) : sE[d * kWThreads + threadIdx.x];
                    fx = e.x;
                    fy = e.y;
                } else {
                    const double zr = -dq * Hx, zi = -dq * Hy;
                    double sn, cs;
                    sincos(zi, &sn, &cs);
                    const double m = exp(zr);
                    fx = m * cs;
                    fy = m * sn;
                }
                const double2 wv = P.w[(size_t)c * MM + parc];
                const double px = S.x * wv.x - S.y * wv.y, py = S.x * wv.y + S.y * wv.x;
                child = make_double2(px * fx - py * fy, px * fy + py * fx);
                return child.x * child.x + child.y * child.y >= P.theta2;
            }
        };
        // pass 1: the survivors of each group, counted; one output range per
        // block and round (a block scan and one atomic), then pass 2 forms
        // the survivors again (the same arithmetic) and writes them
        unsigned long long kmask = 0ull;
        if (valid)
            for (int c = sub; c < MM; c += sub_n) {
                double2 child;
                if (child_of(c, child)) kmask |= 1ull << c;
            }
        const unsigned cnt = (unsigned)__popcll(kmask);
        unsigned inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if ((int)lane >= o) inc += y;
        }
        if (lane == 31) s_wc[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < kWThreads / 32; ++w) {
                const unsigned v = s_wc[w];
                s_wc[w] = (unsigned)tot;
                tot += v;
            }
            s_base = tot ? atomicAdd(&st->n_out, tot) : 0ull;
        }
        __syncthreads();
        unsigned long long o = s_base + s_wc[threadIdx.x >> 5] + (inc - cnt);
        __syncthreads();   // s_wc and s_base are rewritten in the next round
        if (cnt && (long long)(o + cnt) > P.max_paths) {
            atomicOr(&st->err, kWErrPaths);
            kmask = 0ull;
        }
        for (unsigned long long m = kmask; m; m &= m - 1ull, ++o) {
            const int c = __ffsll((long long)m) - 1;
            double2 child;
            child_of(c, child);
            P.klo[outp][o] = clo | (unsigned long long)((c / M) | ((c % M) << 4));
            P.khi[outp][o] = chi;
            if constexpr (C64) static_cast<float2 *>(P.amps[outp])[o] = make_float2((float)child.x, (float)child.y);
            else static_cast<double2 *>(P.amps[outp])[o] = child;
        }
    }
}

// rho(t+1) by newest point from the appended children: per-block FP64 sums
__global__ void __launch_bounds__(kWThreads) k_w_rho(WParams P) {
    __shared__ double2 s_r[kWMaxMM];
    WState *st = P.st;
    const int MM = P.M * P.M;
    for (int k = threadIdx.x; k < MM; k += blockDim.x) s_r[k] = make_double2(0.0, 0.0);
    __syncthreads();
    if (!st->err) {
        const int outp = (int)((st->t + 1) & 1);
        const unsigned long long n = min(st->n_out, (unsigned long long)P.max_paths);
        for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
             i += (unsigned long long)gridDim.x * blockDim.x) {
            const unsigned v = (unsigned)(P.klo[outp][i] & 0xffull);
            const double2 a = amp_of(P, P.amps[outp], i);
            const int k = (int)(v & 15u) * P.M + (int)(v >> 4);
            atomicAdd(&s_r[k].x, a.x);
            atomicAdd(&s_r[k].y, a.y);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < MM; k += blockDim.x) P.rho_part[(size_t)blockIdx.x * MM + k] = s_r[k];
}

// one block: rho(t+1) from the block sums, the step's record, the new state
__global__ void k_w_finalize(WParams P, int nblk, int merge) {
    WState *st = P.st;
    const int MM = P.M * P.M;
    if (st->err) return;
    const unsigned long long tn = st->t + 1;
    const size_t slot = (size_t)(tn % (unsigned long long)P.rho_hist);
    for (int k = threadIdx.x; k < MM; k += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double2 v = P.rho_part[(size_t)b * MM + k];
            x += v.x;
            y += v.y;
        }
        P.rho_ring[slot * MM + k] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long groups = merge ? st->n_groups : st->n_cur;
        WRec r;
        r.t = (long long)tn;
        r.groups = (long long)groups;
        r.extended = (long long)groups * MM;
        r.kept = (long long)st->n_out;
        r.inter = r.kept;
        P.stats[slot] = r;
        st->n_cur = st->n_out;
        st->t = tn;
        st->n_groups = 0;
        st->n_out = 0;
    }
}

// history tables: T[n_act][j][v] = eta_{j+1} q[forward] - conj(eta_{j+1})
// q[backward] for the point at byte j of a key while n_act points are held
// (bytes past the history contribute nothing)
__global__ void k_w_build_lut(double2 *lut, float2 *lutf, float2 *lutlo, const double2 *eta, const double *q, int M,
                              int dkmax) {
    const int nb = dkmax - 1, total = dkmax * nb * 256;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int v = i % 256, j = (i / 256) % nb, n_act = i / (256 * nb) + 1;
        const int sp = v & 15, sm = v >> 4;
        double hx = 0.0, hy = 0.0;
        if (j <= n_act - 2 && sp < M && sm < M) {
            const double2 e = eta[j + 1];
            hx = e.x * q[sp] - e.x * q[sm];
            hy = e.y * q[sp] + e.y * q[sm];
        }
        lut[i] = make_double2(hx, hy);
        const float fx = (float)hx, fy = (float)hy;
        lutf[i] = make_float2(fx, fy);
        lutlo[i] = make_float2((float)(hx - (double)fx), (float)(hy - (double)fy));
    }
}

// W[(a,b)][(a',b')] = U[a,a'] conj(U[b,b']) exp(-(q_a - q_b)(eta_0 q_a - conj(eta_0) q_b))
__global__ void k_w_build_w(double2 *w, float4 *wf, const double2 *U, const double2 *eta, const double *q, int M) {
    const int MM = M * M;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MM * MM; i += gridDim.x * blockDim.x) {
        const int child = i / MM, par = i % MM;
        const int a = child / M, b = child % M, ap = par / M, bp = par % M;
        const double2 ua = U[a * M + ap], ub = U[b * M + bp];
        const double2 prop = make_double2(ua.x * ub.x + ua.y * ub.y, ua.y * ub.x - ua.x * ub.y);
        const double dq = q[a] - q[b];
        const double2 e0 = eta[0];
        const double zr = -dq * (e0.x * q[a] - e0.x * q[b]), zi = -dq * (e0.y * q[a] + e0.y * q[b]);
        double s, c;
        sincos(zi, &s, &c);
        const double m = exp(zr);
        const double2 f = make_double2(m * c, m * s);
        const double2 v = make_double2(prop.x * f.x - prop.y * f.y, prop.x * f.y + prop.y * f.x);
        w[i] = v;
        const float hx = (float)v.x, hy = (float)v.y;
        wf[i] = make_float4(hx, hy, (float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
}

__global__ void k_w_clear_table(WSlot *slots, unsigned long long *ttie, unsigned long long n) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        WSlot fresh;
        fresh.gk = kWEmpty;
        fresh.wm = 0ull;
        fresh.sre = fresh.sim = 0.0;
        slots[i] = fresh;
        ttie[i] = kWEmpty;
    }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct WLayout {
    size_t klo[2], khi[2], amps[2], slot_of, groups, trep, slots, ttie, lut, lutf, lutlo, w, wf, U, eta, q,
        rho_part, rho, stats, state, total;
    unsigned long long tcap;
};

const char *wide_invalid(const qp_config *c) {
    if (!c) return "null config";
    if (c->M < 2 || c->M > kWMaxM) return "M out of range (2..8)";
    if (c->dkmax < 1 || c->dkmax > kWMaxDk) return "dkmax out of range (1..16)";
    if (!(c->dt > 0.0) || !std::isfinite(c->dt)) return "dt must be positive";
    if (!(c->theta >= 0.0) || !std::isfinite(c->theta)) return "theta must be >= 0";
    if (c->precision != QP_FP64 && c->precision != QP_C64) return "unknown precision";
    if (c->max_paths < 16 || c->max_paths > (1ll << 32)) return "max_paths out of range (16 .. 2^32)";
    if (c->max_groups < 0 || c->max_groups > (1ll << 32)) return "max_groups out of range";
    if (c->rho_history < 0 || c->rho_history > (1 << 20)) return "rho_history out of range";
    if (c->n_inst > 1) return "wide keys take single problems only";
    if (c->scheme != QP_PREMERGE) return "wide keys take the pre-merging order only";
    if (!c->q || !c->hs_re) return "q and hs required";
    for (int i = 0; i < c->M; ++i)
        if (!std::isfinite(c->q[i])) return "q must be finite";
    return nullptr;
}

WLayout wide_layout(const qp_config *c) {
    WLayout L{};
    const long long mp = c->max_paths;
    const long long mg = c->max_groups ? c->max_groups : mp;
    unsigned long long tcap = 16;
    while (tcap < 2ull * (unsigned long long)mg) tcap <<= 1;
    L.tcap = tcap;
    const int MM = c->M * c->M, R = c->rho_history ? c->rho_history : 4096;
    const size_t ab = c->precision == QP_C64 ? 8 : 16;
    const size_t nlut = (size_t)c->dkmax * std::max(1, c->dkmax - 1) * 256;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = a256(off + bytes); return o; };
    L.state = take(sizeof(WState));
    for (int k = 0; k < 2; ++k) {
        L.klo[k] = take(mp * 8);
        L.khi[k] = take(mp * 8);
        L.amps[k] = take(mp * ab);
    }
    L.slot_of = take(mp * 4);
    L.groups = take(mg * 4);
    L.trep = take(tcap * 4);
    L.slots = take(tcap * sizeof(WSlot));
    L.ttie = take(tcap * 8);
    L.lut = take(nlut * 16);
    L.lutf = take(nlut * 8);
    L.lutlo = take(nlut * 8);
    L.w = take((size_t)MM * MM * 16);
    L.wf = take((size_t)MM * MM * 16);
    L.U = take((size_t)MM * 16);
    L.eta = take((size_t)c->dkmax * 16);
    L.q = take((size_t)c->M * 8);
    L.rho_part = take((size_t)2048 * MM * 16);
    L.rho = take((size_t)R * MM * 16);
    L.stats = take((size_t)R * sizeof(WRec));
    L.total = off;
    return L;
}

}  // namespace

struct qp_wide {
    qp_config cfg;
    std::vector<double> q;
    std::vector<qp::cplx> hs, U;
    std::vector<int> mask;
    WLayout L;
    WParams P{};
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    int nsm = 0, nblk = 0;
    bool have_eta = false, have_state = false, failed = false;
    std::string err;
};

namespace {

qp_status wfail(qp_wide *w, qp_status s, const std::string &msg) {
    if (w) w->err = msg;
    return s;
}
#define QW_CUDA(w, call)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return wfail((w), QP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

qp_status wide_set_mask_params(qp_wide *w, const std::vector<int> &P) {
    const int dk = w->cfg.dkmax;
    std::vector<char> in(dk, 0);
    in[0] = 1;
    for (int p : P)
        if (p >= 1) in[p - 1] = 1;
    int np = 0, nc = 0;
    for (int p = 0; p < dk; ++p) {
        if (in[p]) w->P.pp[np++] = p;
        else w->P.co[nc++] = p;
    }
    if (6 * np > 64) return wfail(w, QP_ERR_ARG, "wide keys: P' may hold at most 10 positions (64-bit group key)");
    if (6 * nc > 64) return wfail(w, QP_ERR_ARG, "wide keys: at most 10 positions outside P' (64-bit tie key)");
    w->P.npp = np;
    w->P.nco = nc;
    return QP_OK;
}

qp_status wide_read_state(qp_wide *w, WState *s) {
    QW_CUDA(w, cudaMemcpyAsync(s, w->P.st, sizeof(WState), cudaMemcpyDeviceToHost, w->stream));
    QW_CUDA(w, cudaStreamSynchronize(w->stream));
    if (s->err) {
        w->failed = true;
        std::string what;
        if (s->err & kWErrPaths) what += " path buffer (max_paths)";
        if (s->err & kWErrGroups) what += " merge groups (max_groups)";
        if (s->err & kWErrProbe) what += " merge table probe limit";
        return wfail(w, QP_ERR_CAPACITY, "capacity exceeded at step " + std::to_string(s->t + 1) + ":" + what);
    }
    return QP_OK;
}

}  // namespace

extern "C" {

qp_status qp_wide_workspace_size(const qp_config *cfg, size_t *bytes) {
    if (!bytes || wide_invalid(cfg)) return QP_ERR_ARG;
    *bytes = wide_layout(cfg).total;
    return QP_OK;
}

qp_status qp_wide_create(const qp_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream, qp_wide **out) {
    if (!out) return QP_ERR_ARG;
    *out = nullptr;
    if (wide_invalid(cfg) || !d_workspace) return QP_ERR_ARG;
    const WLayout L = wide_layout(cfg);
    if (bytes < L.total) return QP_ERR_OOM;
    qp_wide *w = new (std::nothrow) qp_wide;
    if (!w) return QP_ERR_OOM;
    w->cfg = *cfg;
    w->q.assign(cfg->q, cfg->q + cfg->M);
    const int M = cfg->M, MM = M * M;
    w->hs.resize(MM);
    for (int i = 0; i < MM; ++i) w->hs[i] = qp::cplx(cfg->hs_re[i], cfg->hs_im ? cfg->hs_im[i] : 0.0);
    w->cfg.q = nullptr;
    w->cfg.hs_re = w->cfg.hs_im = nullptr;
    w->U = qp::short_time_propagator(M, w->hs, cfg->dt);
    w->L = L;
    w->ws = static_cast<char *>(d_workspace);
    w->stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&w->nsm, cudaDevAttrMultiProcessorCount, dev);
    w->nblk = std::min(2048, std::max(1, w->nsm) * 4);
    WParams &P = w->P;
    P.M = M;
    P.dkmax = cfg->dkmax;
    P.c64 = cfg->precision == QP_C64 ? 1 : 0;
    P.rho_hist = cfg->rho_history ? cfg->rho_history : 4096;
    P.max_paths = cfg->max_paths;
    P.max_groups = cfg->max_groups ? cfg->max_groups : cfg->max_paths;
    P.tcap_mask = L.tcap - 1;
    P.theta2 = cfg->theta * cfg->theta;
    P.theta2f = (float)P.theta2;
    P.tie_rel = cfg->precision == QP_C64 ? 1e-6 : 1e-12;   // the narrow engines' windows (reading R4, R11)
    for (int i = 0; i < M; ++i) P.q[i] = cfg->q[i];
    P.ndelta = 0;
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
            const double d = cfg->q[a] - cfg->q[b];   // as the kernel forms it
            int k = -1;
            if (d != 0.0) {
                for (int j = 0; j < P.ndelta; ++j)
                    if (P.delta[j] == d) k = j;
                if (k < 0) {
                    k = P.ndelta;
                    P.delta[P.ndelta++] = d;
                }
            }
            P.dsel[a * M + b] = (signed char)k;
        }
    char *ws = w->ws;
    for (int k = 0; k < 2; ++k) {
        P.klo[k] = reinterpret_cast<unsigned long long *>(ws + L.klo[k]);
        P.khi[k] = reinterpret_cast<unsigned long long *>(ws + L.khi[k]);
        P.amps[k] = ws + L.amps[k];
    }
    P.slot_of = reinterpret_cast<unsigned *>(ws + L.slot_of);
    P.groups = reinterpret_cast<unsigned *>(ws + L.groups);
    P.trep = reinterpret_cast<unsigned *>(ws + L.trep);
    P.slots = reinterpret_cast<WSlot *>(ws + L.slots);
    P.ttie = reinterpret_cast<unsigned long long *>(ws + L.ttie);
    P.lut = reinterpret_cast<const double2 *>(ws + L.lut);
    P.lutf = reinterpret_cast<const float2 *>(ws + L.lutf);
    P.lutlo = reinterpret_cast<const float2 *>(ws + L.lutlo);
    P.w = reinterpret_cast<const double2 *>(ws + L.w);
    P.wf = reinterpret_cast<const float4 *>(ws + L.wf);
    P.rho_part = reinterpret_cast<double2 *>(ws + L.rho_part);
    P.rho_ring = reinterpret_cast<double2 *>(ws + L.rho);
    P.stats = reinterpret_cast<WRec *>(ws + L.stats);
    P.st = reinterpret_cast<WState *>(ws + L.state);
    std::vector<int> full(cfg->dkmax);
    for (int p = 0; p < cfg->dkmax; ++p) full[p] = p;
    w->mask = full;
    if (wide_set_mask_params(w, full) != QP_OK && cfg->dkmax > 0) {
        // the full mask of a long window does not fit a 64-bit group key:
        // a mask must be set before qp_wide_set_rho0
        w->P.npp = -1;
    }
    if (cudaFuncSetAttribute(k_w_expand<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kWMaxTabDelta * kWThreads * 16) != cudaSuccess ||
        cudaFuncSetAttribute(k_w_expand<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kWMaxTabDelta * kWThreads * 8) != cudaSuccess) {
        delete w;
        return QP_ERR_CUDA;
    }
    *out = w;
    return QP_OK;
}

void qp_wide_destroy(qp_wide *w) { delete w; }

qp_status qp_wide_set_eta(qp_wide *w, const double *re, const double *im, int n) {
    if (!w) return QP_ERR_ARG;
    const int dk = w->cfg.dkmax, M = w->cfg.M, MM = M * M;
    if (!re || !im || n < dk) return wfail(w, QP_ERR_ARG, "need dkmax coefficients");
    std::vector<double2> e(dk), Ud(MM);
    for (int i = 0; i < dk; ++i) {
        if (!std::isfinite(re[i]) || !std::isfinite(im[i])) return wfail(w, QP_ERR_ARG, "eta must be finite");
        e[i] = make_double2(re[i], im[i]);
    }
    for (int i = 0; i < MM; ++i) Ud[i] = make_double2(w->U[i].real(), w->U[i].imag());
    char *ws = w->ws;
    QW_CUDA(w, cudaMemcpyAsync(ws + w->L.eta, e.data(), dk * sizeof(double2), cudaMemcpyHostToDevice, w->stream));
    QW_CUDA(w, cudaMemcpyAsync(ws + w->L.U, Ud.data(), MM * sizeof(double2), cudaMemcpyHostToDevice, w->stream));
    QW_CUDA(w, cudaMemcpyAsync(ws + w->L.q, w->q.data(), M * sizeof(double), cudaMemcpyHostToDevice, w->stream));
    if (dk >= 2)
        k_w_build_lut<<<64, 256, 0, w->stream>>>(reinterpret_cast<double2 *>(ws + w->L.lut),
                                                 reinterpret_cast<float2 *>(ws + w->L.lutf),
                                                 reinterpret_cast<float2 *>(ws + w->L.lutlo),
                                                 reinterpret_cast<const double2 *>(ws + w->L.eta),
                                                 reinterpret_cast<const double *>(ws + w->L.q), M, dk);
    k_w_build_w<<<16, 256, 0, w->stream>>>(reinterpret_cast<double2 *>(ws + w->L.w),
                                           reinterpret_cast<float4 *>(ws + w->L.wf),
                                           reinterpret_cast<const double2 *>(ws + w->L.U),
                                           reinterpret_cast<const double2 *>(ws + w->L.eta),
                                           reinterpret_cast<const double *>(ws + w->L.q), M);
    QW_CUDA(w, cudaGetLastError());
    QW_CUDA(w, cudaStreamSynchronize(w->stream));   // e, Ud are host temporaries
    w->have_eta = true;
    return QP_OK;
}

qp_status qp_wide_set_mask(qp_wide *w, const int *positions, int n) {
    if (!w) return QP_ERR_ARG;
    const int dk = w->cfg.dkmax;
    std::vector<int> P;
    if (!positions || n == 0) {
        for (int p = 0; p < dk; ++p) P.push_back(p);
    } else {
        for (int i = 0; i < n; ++i) {
            if (positions[i] < 0 || positions[i] >= dk) return wfail(w, QP_ERR_ARG, "mask position out of range");
            P.push_back(positions[i]);
        }
    }
    std::sort(P.begin(), P.end());
    P.erase(std::unique(P.begin(), P.end()), P.end());
    if (P.empty() || P[0] != 0 || (dk >= 2 && (P.size() < 2 || P[1] != 1)))
        return wfail(w, QP_ERR_ARG, "mask must contain positions 0 and 1");
    const WParams keep = w->P;
    const qp_status s = wide_set_mask_params(w, P);
    if (s != QP_OK) {
        w->P = keep;
        return s;
    }
    w->mask = P;
    return QP_OK;
}

qp_status qp_wide_set_rho0(qp_wide *w, const double *re, const double *im) {
    if (!w) return QP_ERR_ARG;
    if (!re) return wfail(w, QP_ERR_ARG, "rho0 required");
    if (!w->have_eta) return wfail(w, QP_ERR_STATE, "qp_wide_set_eta must come before qp_wide_set_rho0");
    if (w->P.npp < 0) return wfail(w, QP_ERR_STATE, "set a mask whose P' fits the 64-bit group key first");
    const int M = w->cfg.M, MM = M * M;
    std::vector<unsigned long long> lo, hi;
    std::vector<double2> amps, rho(MM);
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
            const double x = re[a * M + b], y = im ? im[a * M + b] : 0.0;
            if (!std::isfinite(x) || !std::isfinite(y)) return wfail(w, QP_ERR_ARG, "rho0 must be finite");
            rho[a * M + b] = make_double2(x, y);
            if (x != 0.0 || y != 0.0) {
                lo.push_back((unsigned long long)(a | (b << 4)));
                hi.push_back(0ull);
                amps.push_back(make_double2(x, y));
            }
        }
    const size_t n = lo.size();
    std::vector<float2> af(n);
    for (size_t i = 0; i < n; ++i) af[i] = make_float2((float)amps[i].x, (float)amps[i].y);
    const size_t ab = w->P.c64 ? 8 : 16;
    QW_CUDA(w, cudaMemcpyAsync(w->P.klo[0], lo.data(), n * 8, cudaMemcpyHostToDevice, w->stream));
    QW_CUDA(w, cudaMemcpyAsync(w->P.khi[0], hi.data(), n * 8, cudaMemcpyHostToDevice, w->stream));
    QW_CUDA(w, cudaMemcpyAsync(w->P.amps[0], w->P.c64 ? (const void *)af.data() : (const void *)amps.data(), n * ab,
                               cudaMemcpyHostToDevice, w->stream));
    WState s{};
    s.n_cur = n;
    QW_CUDA(w, cudaMemcpyAsync(w->P.st, &s, sizeof(WState), cudaMemcpyHostToDevice, w->stream));
    QW_CUDA(w, cudaMemcpyAsync(w->P.rho_ring, rho.data(), MM * sizeof(double2), cudaMemcpyHostToDevice, w->stream));
    WRec r0{0, 0, 0, (long long)n, (long long)n};
    QW_CUDA(w, cudaMemcpyAsync(w->P.stats, &r0, sizeof(WRec), cudaMemcpyHostToDevice, w->stream));
    k_w_clear_table<<<std::max(1, w->nsm) * 4, 256, 0, w->stream>>>(w->P.slots, w->P.ttie,
                                                                    w->L.tcap);
    QW_CUDA(w, cudaGetLastError());
    QW_CUDA(w, cudaStreamSynchronize(w->stream));
    w->have_state = true;
    w->failed = false;
    return QP_OK;
}

qp_status qp_wide_step(qp_wide *w, int nsteps) {
    if (!w) return QP_ERR_ARG;
    if (nsteps < 0) return wfail(w, QP_ERR_ARG, "nsteps < 0");
    if (!w->have_state) return wfail(w, QP_ERR_STATE, "qp_wide_set_rho0 must come before qp_wide_step");
    if (w->failed) return wfail(w, QP_ERR_STATE, "context holds a device error; call qp_wide_set_rho0");
    if (nsteps == 0) return QP_OK;
    // the step count on the host decides merge or fill: read t once
    WState s;
    qp_status r = wide_read_state(w, &s);
    if (r != QP_OK) return r;
    unsigned long long t = s.t;
    const int g = w->nblk;
    const int MMh = w->cfg.M * w->cfg.M;
    // lanes per group in the expansion: complex64 is latency-bound (shorter
    // chains per lane pay for the repeated per-group set-up); FP64 is bound
    // by its pipe (1/64 of FP32), where the repeated set-up would cost more
    const int sub_n = !w->P.c64 ? 1 : (MMh >= 32 ? 4 : (MMh >= 16 ? 2 : 1));
    for (int k = 0; k < nsteps; ++k, ++t) {
        const int merge = t + 1 >= (unsigned long long)w->cfg.dkmax ? 1 : 0;
        if (merge) {
            k_w_insert<<<g, kWThreads, 0, w->stream>>>(w->P);
            k_w_tie<false><<<g, kWThreads, 0, w->stream>>>(w->P);
            k_w_tie<true><<<g, kWThreads, 0, w->stream>>>(w->P);
        }
        const bool tab = w->P.ndelta <= kWMaxTabDelta;
        const size_t tsm = tab ? (size_t)w->P.ndelta * kWThreads * (w->P.c64 ? 8 : 16) : 0;
        if (w->P.c64) {
            if (tab) k_w_expand<true, true><<<g, kWThreads, tsm, w->stream>>>(w->P, merge, sub_n);
            else k_w_expand<true, false><<<g, kWThreads, 0, w->stream>>>(w->P, merge, sub_n);
        } else {
            if (tab) k_w_expand<false, true><<<g, kWThreads, tsm, w->stream>>>(w->P, merge, sub_n);
            else k_w_expand<false, false><<<g, kWThreads, 0, w->stream>>>(w->P, merge, sub_n);
        }
        k_w_rho<<<g, kWThreads, 0, w->stream>>>(w->P);
        k_w_finalize<<<1, 64, 0, w->stream>>>(w->P, g, merge);
        QW_CUDA(w, cudaGetLastError());
    }
    return QP_OK;
}

qp_status qp_wide_current(qp_wide *w, int64_t *t, int64_t *n) {
    if (!w) return QP_ERR_ARG;
    if (!w->have_state) return wfail(w, QP_ERR_STATE, "no state");
    WState s;
    const qp_status r = wide_read_state(w, &s);
    if (t) *t = (int64_t)s.t;
    if (n) *n = (int64_t)s.n_cur;
    return r;
}

qp_status qp_wide_read_rho(qp_wide *w, int64_t t0, int count, double *re, double *im) {
    if (!w) return QP_ERR_ARG;
    if (!re || !im || count < 0) return wfail(w, QP_ERR_ARG, "bad output");
    if (!w->have_state) return wfail(w, QP_ERR_STATE, "no state");
    WState s;
    qp_status r = wide_read_state(w, &s);
    if (r != QP_OK) return r;
    const int MM = w->cfg.M * w->cfg.M;
    const int64_t R = w->P.rho_hist;
    if (t0 < 0 || t0 + count - 1 > (int64_t)s.t || (int64_t)s.t - t0 >= R) return wfail(w, QP_ERR_ARG, "t outside the kept history");
    std::vector<double2> buf((size_t)MM);
    for (int k = 0; k < count; ++k) {
        const int64_t t = t0 + k;
        QW_CUDA(w, cudaMemcpyAsync(buf.data(), w->P.rho_ring + (size_t)(t % R) * MM, MM * sizeof(double2),
                                   cudaMemcpyDeviceToHost, w->stream));
        QW_CUDA(w, cudaStreamSynchronize(w->stream));
        for (int i = 0; i < MM; ++i) {
            re[(size_t)k * MM + i] = buf[i].x;
            im[(size_t)k * MM + i] = buf[i].y;
        }
    }
    return QP_OK;
}

qp_status qp_wide_read_stats(qp_wide *w, int64_t t0, int count, qp_step_stats *out) {
    if (!w) return QP_ERR_ARG;
    if (!out || count < 0) return wfail(w, QP_ERR_ARG, "bad output");
    WState s;
    qp_status r = wide_read_state(w, &s);
    if (r != QP_OK) return r;
    const int64_t R = w->P.rho_hist;
    if (t0 < 0 || t0 + count - 1 > (int64_t)s.t || (int64_t)s.t - t0 >= R) return wfail(w, QP_ERR_ARG, "t outside the kept history");
    for (int k = 0; k < count; ++k) {
        WRec rec;
        QW_CUDA(w, cudaMemcpyAsync(&rec, w->P.stats + (size_t)((t0 + k) % R), sizeof(WRec), cudaMemcpyDeviceToHost,
                                   w->stream));
        QW_CUDA(w, cudaStreamSynchronize(w->stream));
        out[k].t = rec.t;
        out[k].groups = rec.groups;
        out[k].extended = rec.extended;
        out[k].kept = rec.kept;
        out[k].intermediate = rec.inter;
    }
    return QP_OK;
}

qp_status qp_wide_export_paths(qp_wide *w, uint64_t *keys, double *amps, int64_t cap, int64_t *n) {
    if (!w) return QP_ERR_ARG;
    if (!n || cap < 0 || (cap > 0 && (!keys || !amps))) return wfail(w, QP_ERR_ARG, "bad output");
    if (!w->have_state) return wfail(w, QP_ERR_STATE, "no state");
    WState s;
    qp_status r = wide_read_state(w, &s);
    if (r != QP_OK) return r;
    *n = (int64_t)s.n_cur;
    if ((int64_t)s.n_cur > cap) return wfail(w, QP_ERR_CAPACITY, "export buffer too small");
    const int buf = (int)(s.t & 1);
    const size_t cnt = s.n_cur;
    std::vector<unsigned long long> lo(cnt), hi(cnt);
    std::vector<float2> af(w->P.c64 ? cnt : 0);
    std::vector<double2> ad(w->P.c64 ? 0 : cnt);
    QW_CUDA(w, cudaMemcpyAsync(lo.data(), w->P.klo[buf], cnt * 8, cudaMemcpyDeviceToHost, w->stream));
    QW_CUDA(w, cudaMemcpyAsync(hi.data(), w->P.khi[buf], cnt * 8, cudaMemcpyDeviceToHost, w->stream));
    if (w->P.c64)
        QW_CUDA(w, cudaMemcpyAsync(af.data(), w->P.amps[buf], cnt * 8, cudaMemcpyDeviceToHost, w->stream));
    else
        QW_CUDA(w, cudaMemcpyAsync(ad.data(), w->P.amps[buf], cnt * 16, cudaMemcpyDeviceToHost, w->stream));
    QW_CUDA(w, cudaStreamSynchronize(w->stream));
    for (size_t i = 0; i < cnt; ++i) {
        keys[2 * i] = lo[i];
        keys[2 * i + 1] = hi[i];
        amps[2 * i] = w->P.c64 ? af[i].x : ad[i].x;
        amps[2 * i + 1] = w->P.c64 ? af[i].y : ad[i].y;
    }
    return QP_OK;
}

const char *qp_wide_last_error(const qp_wide *w) { return w ? w->err.c_str() : "null context"; }

}  // extern "C"
