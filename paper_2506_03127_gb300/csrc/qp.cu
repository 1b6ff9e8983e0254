// libqp: GB300 (sm_103a) kernels and C ABI of the MACGIC-iQUAPI path update.
//
// One propagation step Omega(t-1) -> Omega(t) (paper Sec. 3.1, routines
// premerging() and propagation()).  Three engines compute it:
//   stream engine (the default where the mask allows it): the stored set
//     kept sorted in M^2 regions by newest point, so that every pre-merge
//     group is a run; k_stream_step (tiles, segmented group sums, survivors
//     compacted in order by a decoupled look-back), k_stream_regular (the
//     unfiltered full-memory step as a streaming map) and k_stream_batch
//     (independent instances in n_inst * M^2 regions);
//   merge-table engine (any mask, the symmetric splitting, sharded steps):
//     the kernels listed below;
//   post-merging engine (the order of Sec. 2.1): k_post_*, a device radix
//     sort (k_rs_*) and a reduction by key (k_rbk_*).
// Also here: the partition of a stored set by owner rank (k_part_*), the
// allocation-free step (qp_step_noalloc) and the C ABI.  Every kernel reads
// the step index and the path counts from a small device-resident state
// block, so the host never waits on a count and one captured CUDA graph
// replays any step.  The merge-table engine's sequence:
//
//   k_insert    pre-merge pass 1 (window full only): each stored path
//               inserts its masked key into the merge table (open
//               addressing, atomicCAS claim), adds its amplitude into the
//               group sum (FP64 atomics) and raises the group's maximum
//               |amp|^2 (atomicMax on the FP64 bit pattern; non-negative
//               doubles order like uint64).
//   k_tiebreak  pre-merge pass 2: paths whose |amp|^2 is within the tie
//               window of the group maximum (1e-12 relative in FP64, 1e-6
//               in complex64) compete for the representative
//               with atomicMin on the packed key (deterministic choice
//               among equal weights).
//   k_expand    per group (or per stored path while the window fills): the
//               history part H of the influence exponent from per-byte
//               lookup tables, the M^2 children weighted by
//               U[a,a'] conj(U[b,b']) exp(-(q_a-q_b)(H + eta_0 q_a - eta_0* q_b)),
//               filter |amp|^2 >= theta^2, rho(t) accumulated in registers
//               then reduced per block, survivors appended to the other
//               ping-pong buffer (warp-aggregated atomic cursor).  The
//               group's table slot is reset after it is read.
//   k_finalize  one thread: publishes the new count, per-step statistics,
//               advances t, zeroes the next rho accumulator.
//
// Precision (template parameter Amp): double2 amplitudes (QP_FP64) or
// float2 amplitudes (QP_C64) with the influence exponent accumulated in FP32
// with compensated (Kahan) sums.  On the C64 path eta and rho stay FP64; the
// group sums are FP64 atomic sums in the merge table (k_insert), while the
// stream kernels add a group's FP32 members in FP32 with the rounding error
// of every addition kept in a second word (TwoSum) and round the pair once
// to FP32, the precision the children are formed in.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned int kNoSlot = 0xffffffffu;
constexpr int kMaxRuns = 8;
constexpr int kMaxProbe = 64;
constexpr unsigned int kErrPaths = 1u, kErrGroups = 2u, kErrProbe = 4u, kErrTimeout = 8u;
constexpr int kLutEntries = 256;
constexpr int kInsertThreads = 256;
constexpr int kExpandThreads = 128;
constexpr int kMaxExpandBlocks = 2048;
constexpr int kPersistThreads = 256;
constexpr int kMaxInst = 128;                      // instances of one batched context
constexpr int kStreamMinTile = 256;                 // smallest stream tile (256, 512 or 1024 stored paths)
constexpr int kRegThreads = 256;                    // threads per block of the regular stream kernel
constexpr int kStreamWarps = 8;                     // warps per block of both stream kernels (256 threads)
constexpr size_t kMaxStreamLut = 32 * 1024;         // history tables staged in shared memory up to this size
constexpr int kStreamThreads = 256;
constexpr unsigned kLbAgg = 1u, kLbInc = 2u;        // look-back word states (bits 30-31)
constexpr long long kBarrierCycles = 4000000000ll;  // ~2 s at 2 GHz: a grid barrier gives up after this
constexpr int kMaxDelta = 12;
constexpr double kTieRelFP64 = 1e-12;  // weights equal to this relative width are ties (R4)
constexpr double kTieRelC64 = 1e-6;    // same, at complex64 resolution (about 17 units in the last place of |amp|^2)

struct __align__(32) Slot {
    unsigned long long mk;     // masked key, kEmpty when free
    unsigned long long wmax;   // bit pattern of max |amp|^2 (FP64; FP32 on the C64 path)
    double sre, sim;           // FP64 group sum
};

struct __align__(128) DevState {
    unsigned long long t;             // time index of the stored set Omega(t)
    unsigned long long n_cur;         // stored paths in buffer (t & 1)
    unsigned long long cnt_groups[3]; // step t' uses [t' % 3]: merge groups claimed
    unsigned long long cnt_out[3];    // step t' uses [t' % 3]: survivors appended
    unsigned int err;                 // error bits, sticky until qp_set_rho0
    unsigned int stall_tile;          // test hook: tile ticket + 1 whose look-back words are withheld (0: none)
    unsigned long long err_t;         // step at which the error was raised
    unsigned int ticket[3];           // stream engine: tile tickets, step t' uses [t' % 3]
    unsigned int pad0;
    unsigned long long reg_done;      // stream engine: tn + 1 when the regular kernel took step tn, else 0
    unsigned long long rho_pending;   // stream engine: step whose block partials of rho are not summed yet (0: none)
    unsigned int rho_nblk;            // ... and the blocks that wrote them
    unsigned int post_bits;           // post-merging: significant bits of the running step's sort key
    unsigned long long post_n;        // post-merging: unmerged children of the running step
    unsigned long long scan_total;    // total of the last multi-block scan
    unsigned int bar_count;           // grid barrier of the persistent kernel: arrivals
    unsigned int pad1[31];
    unsigned int bar_gen;             // generation (own cache line)
    unsigned int pad2[31];
};

struct StepRec { long long t, groups, extended, kept, inter; };

struct Params {
    int M, bs, b, dkmax;
    int nchunks;                       // bytes of the history part of a key
    int dense;                         // 1: table index = compressed masked key
    int nruns;
    int run_shift[kMaxRuns];
    int run_off[kMaxRuns];
    unsigned long long run_mask[kMaxRuns];
    unsigned long long pmask;          // bits of the pre-merge positions P'
    unsigned int tcap_log2;
    unsigned long long tcap_mask;
    double theta2;
    long long max_paths, max_groups;
    int rho_hist;
    unsigned long long *keys[2];
    void *amps[2];
    Slot *slots;
    unsigned long long *repk;
    unsigned int *slot_of;
    unsigned int *groups;
    const double2 *lut;                // [dkmax][nchunks][256] FP64 history tables
    const float2 *lutf;                // same, FP32 hi part
    const float2 *lutf_lo;             // FP32 residual (hi + lo = FP64 value)
    const double2 *wtab;               // [M*M child][M*M parent newest] propagator x new-point influence
    const float4 *wtabf;               // same, FP32 pairs: (hi.x, hi.y, lo.x, lo.y), hi + lo = the FP64 value
    const double2 *etab;               // [dkmax][ndelta][nchunks][256] exp(-delta_d T) tables (FP64 path)
    int ndelta;                        // distinct nonzero q_a - q_b
    float deltaf[12];                  // their values (FP32 path)
    // symmetric Trotter splitting (merge-table engine, single problems):
    // history tables with point 0 on its half interval, and for rho(t) the
    // newest point's end-point correction: tables of the coefficient
    // differences and the per-child half-interval factor (wEt)
    int sym;
    const double2 *lutE;
    const float2 *lutEf, *lutElo;
    const double2 *etabE;
    const double2 *wEt;                // [M*M child][M*M parent], the same for every parent
    const float4 *wEtf;
    int qeq;                           // 1: q equally spaced, q_a = q_0 + a s (s != 0)
    int d_pos, d_neg;                  // ... indices of +s and -s among the differences
    float qstepf;                      // ... s (FP32 path)
    signed char dsel[16];              // child k -> delta index, -1 when q_a == q_b
    float theta2f;
    double tie_rel;                    // relative window of equal weights (R4)
    double2 *rho_ring;                 // [rho_hist][n_inst][M*M]
    double2 *rho_part;                 // [2 (step parity)][kMaxExpandBlocks][n_inst][M*M + 1] per-block partials
    float4 *spart;                     // stream engine: [2][kMaxExpandBlocks][M*M] per-block partials (FP32 pairs)
    long long *scount;                 // stream engine: [2][kMaxExpandBlocks] children written per block
                                       // of rho(t) per instance; element M*M holds the survivor count
    long long *inst_kept;              // [rho_hist][n_inst] stored paths per instance after each step
    unsigned int *fin_count;           // blocks of k_finalize that are done (last one updates the state)
    int n_inst;                        // independent instances (1 = single problem)
    int inst_shift;                    // key bit where the instance index starts (b * dkmax)
    unsigned long long instmask;       // key bits of the instance index
    size_t lut_stride, etab_stride;    // per-instance strides of the history / exp tables (entries)
    // stream engine (stored set kept in M*M regions by newest point, each
    // sorted lexicographically by the older points)
    int stream;                        // 1: stream layout
    unsigned long long prefmask;       // key bits of the prefix positions 0 .. k-1 of P'
    int x_shift;                       // key bit of the one extra position of P' (NX = 4), else -1
    long long region_cap;              // entries per region
    unsigned long long *reg_n;         // [2 (buffer parity)][n_inst][M*M] stored paths per region (stream engine)
    // regular steps of the stream engine (no filter): while the window fills
    // every stored path is its own group; with the full mask, once all
    // full_n = M^(2 dkmax) keys are stored every group is the M*M values of
    // the oldest point, consecutive in its region.  Either way every child
    // survives and child c of group g goes to entry g of region c.
    int reg_fill, reg_merge;
    unsigned long long full_n;
    unsigned long long *tile_state;    // [M*M][max_tiles] look-back words (a bucket's tiles contiguous)
    long long max_tiles;
    StepRec *stats_ring;               // [rho_hist]
    // post-merging engine (the original order, Sec. 2.1): run_* compress the
    // mask P itself instead of P'
    int post;                          // 1: merge the children after the step
    int post_bits_full;                // bits of the sort key once the window is full
    int post_compress;                 // 1: runs of P packed (b |P| bits); 0: key & pmask itself
    unsigned long long *ckeys;         // [max_paths] unmerged children of the step
    void *camps;
    unsigned long long *skey[2];       // [max_paths] sort keys, by pass parity
    unsigned int *sidx[2];             // [max_paths] child index carried through the sort
    unsigned int *rs_hist;             // [256][chunks] digit counts per chunk, scanned in place
    unsigned int *rs_part;             // block partials of the multi-block scan
    unsigned int *rbk_heads;           // [chunks] run heads per chunk, scanned in place
    DevState *st;
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// float -> double by IEEE-754 fields, exactly, with integer operations only
// (keeps the widening of FP32 values off the FP64 pipe): the sign is kept;
// a normal number keeps its 23 fraction bits (shifted up by 29) and its
// exponent rebiased by 1023 - 127; a subnormal m * 2^-149 is normalised at
// its leading one k (exponent k - 149); infinities and NaNs keep the all-ones
// exponent and the shifted fraction; zeros stay zeros.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits = (unsigned long long)(u >> 31) << 63;
    if (e == 0xffu) {
        bits |= (0x7ffull << 52) | ((unsigned long long)m << 29);
    } else if (e != 0u) {
        bits |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m != 0u) {
        const int k = 31 - __clz((int)m);   // 0 .. 22
        bits |= ((unsigned long long)(k + 874) << 52) | (((unsigned long long)m << (52 - k)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)bits);
}

// Path data and merge-table fields are written by other blocks of the same
// persistent kernel, so they are read through L2 (ld.global.cg), never L1.
// Global memory only (never a shared-memory pointer).
__device__ __forceinline__ double2 load_amp(const double2 *p, unsigned long long i) { return __ldcg(p + i); }
__device__ __forceinline__ double2 load_amp(const float2 *p, unsigned long long i) {
    const float2 v = __ldcg(p + i);
    return make_double2(f2d_exact(v.x), f2d_exact(v.y));
}

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return f2d_exact(v); }
__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
// double -> float by the conversion instruction: two per group cost less
// than the integer rounding that would replace them (measured), unlike the
// widening above, which runs once per stored path
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// s + e += b with the rounding error of the addition carried into e
// (TwoSum, Knuth; six FP32 additions, exact for any FP32 operands).
__device__ __forceinline__ void two_sum_acc(float &s, float &e, float b) {
    const float t = s + b, v = t - s;
    e += (s - (t - v)) + (b - v);
    s = t;
}

// atomicAdd with acquire-release semantics at GPU scope (returns the old value).
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Asynchronous 16-byte global -> shared copy (both addresses 16-byte
// aligned); cp_async_wait_all waits for this thread's copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// 16-byte copy of which only the first src_bytes are read (the rest of the
// destination is zero-filled)
__device__ __forceinline__ void cp_async16_part(void *smem, const void *gmem, unsigned src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}


__device__ __forceinline__ unsigned long long table_index(const Params &P, unsigned long long mk) {
    if (P.dense) {
        unsigned long long idx = 0;
        for (int r = 0; r < P.nruns; ++r) idx |= ((mk >> P.run_shift[r]) & P.run_mask[r]) << P.run_off[r];
        return idx;
    }
    return (mk * 0x9E3779B97F4A7C15ull) >> (64 - P.tcap_log2);
}

__device__ __forceinline__ void raise_err(DevState *st, unsigned int bit) {
    atomicOr(&st->err, bit);
}

// Block-wide append: exclusive offset of each thread's cnt items within the
// block and the block's base in a global array, with one atomicAdd on the
// global cursor per block.  All threads of the block must call it.
struct Append {
    unsigned long long base;
    unsigned excl, total;
};
template <int NT>
__device__ __forceinline__ Append block_append(unsigned cnt, unsigned long long *cursor) {
    constexpr int NW = NT / 32;
    __shared__ unsigned s_w[NW];
    __shared__ unsigned s_tot;
    __shared__ unsigned long long s_base;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned v = lane < (unsigned)NW ? s_w[lane] : 0u;
        unsigned vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, vi, o);
            if ((int)lane >= o) vi += y;
        }
        if (lane < (unsigned)NW) s_w[lane] = vi - v;
        if (lane == 31) {
            s_tot = vi;
            s_base = vi ? atomicAdd(cursor, (unsigned long long)vi) : 0ull;
        }
    }
    __syncthreads();
    Append r;
    r.base = s_base;
    r.total = s_tot;
    r.excl = s_w[warp] + incl - cnt;
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- pre-merge

// Pass 1 over the stored set Omega(t) (n paths): claim the group slot of the
// masked key, add the amplitude into the group sum, raise the group maximum
// of |amp|^2.  Newly claimed slots are appended to the group list.
template <typename Amp, int NT>
__device__ __forceinline__ void phase_insert(const Params &P, unsigned long long t, unsigned long long n,
                                             unsigned long long *cnt_groups) {
    DevState *st = P.st;
    const unsigned long long *keys = P.keys[t & 1];
    const Amp *amps = static_cast<const Amp *>(P.amps[t & 1]);
    const unsigned long long stride = (unsigned long long)gridDim.x * NT;
    for (unsigned long long base = blockIdx.x * (unsigned long long)NT; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        bool claimed = false, found = false;
        unsigned long long h = 0;
        if (i < n) {
            const unsigned long long key = __ldcg(keys + i);
            const double2 a = load_amp(amps, i);
            const unsigned long long mk = key & P.pmask;
            h = table_index(P, mk);
            for (int probe = 0; probe < kMaxProbe; ++probe) {
                const unsigned long long cur = *(volatile unsigned long long *)&P.slots[h].mk;
                if (cur == mk) { found = true; break; }
                if (cur == kEmpty) {
                    const unsigned long long prev = atomicCAS(&P.slots[h].mk, kEmpty, mk);
                    if (prev == kEmpty) { claimed = found = true; break; }
                    if (prev == mk) { found = true; break; }
                }
                h = (h + 1) & P.tcap_mask;
            }
            if (found) {
                atomicAdd(&P.slots[h].sre, a.x);
                atomicAdd(&P.slots[h].sim, a.y);
                // weight |a|^2 as ordered bits: FP32 on the C64 path (as in
                // the stream engine), FP64 otherwise
                unsigned long long wb;
                if constexpr (sizeof(Amp) == sizeof(float2)) {
                    const float ax = (float)a.x, ay = (float)a.y;   // exact: a holds FP32 values
                    wb = __float_as_uint(ax * ax + ay * ay);
                } else {
                    wb = (unsigned long long)__double_as_longlong(a.x * a.x + a.y * a.y);
                }
                atomicMax(&P.slots[h].wmax, wb);
                P.slot_of[i] = (unsigned int)h;
            } else {
                P.slot_of[i] = kNoSlot;
                raise_err(st, kErrProbe);
            }
        }
        const Append ap = block_append<NT>(claimed ? 1u : 0u, cnt_groups);
        if (claimed) {
            const unsigned long long g = ap.base + ap.excl;
            if (g < (unsigned long long)P.max_groups) P.groups[g] = (unsigned int)h;
            else raise_err(st, kErrGroups);
        }
    }
}

// Pass 2: paths whose |amp|^2 lies within the tie window of the group maximum
// compete for the representative with atomicMin on the packed key.
template <typename Amp, int NT>
__device__ __forceinline__ void phase_tiebreak(const Params &P, unsigned long long t, unsigned long long n) {
    const unsigned long long *keys = P.keys[t & 1];
    const Amp *amps = static_cast<const Amp *>(P.amps[t & 1]);
    const unsigned long long stride = (unsigned long long)gridDim.x * NT;
    for (unsigned long long i = blockIdx.x * (unsigned long long)NT + threadIdx.x; i < n; i += stride) {
        const unsigned int h = __ldcg(P.slot_of + i);
        if (h == kNoSlot) continue;
        bool tie;
        if constexpr (sizeof(Amp) == sizeof(float2)) {
            const float2 a = __ldcg(amps + i);
            const float w2 = a.x * a.x + a.y * a.y;
            const float wm = __uint_as_float((unsigned)__ldcg(&P.slots[h].wmax));
            tie = w2 >= (float)(1.0 - P.tie_rel) * wm;
        } else {
            const double2 a = load_amp(amps, i);
            const double w2 = a.x * a.x + a.y * a.y;
            const double wm = __longlong_as_double((long long)__ldcg(&P.slots[h].wmax));
            tie = w2 >= (1.0 - P.tie_rel) * wm;
        }
        if (tie) atomicMin(&P.repk[h], __ldcg(keys + i));
    }
}

template <typename Amp>
__global__ void __launch_bounds__(kInsertThreads) k_insert(Params P) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    if (tn < (unsigned long long)P.dkmax) return;   // window not full: no merge
    phase_insert<Amp, kInsertThreads>(P, t, st->n_cur, &st->cnt_groups[tn % 3]);
}

template <typename Amp>
__global__ void __launch_bounds__(kInsertThreads) k_tiebreak(Params P) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    if (tn < (unsigned long long)P.dkmax) return;
    phase_tiebreak<Amp, kInsertThreads>(P, t, st->n_cur);
}

// ---------------------------------------------------------------- extension

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ unsigned key_byte(unsigned long long k, int j) { return (unsigned)(k >> (8 * j)) & 0xffu; }

// Extension of one group (or one stored path while the window fills) to its
// M^2 children.  The influence factor of child (a,b) is
//   exp(-(q_a - q_b)(H + eta_0 q_a - eta_0* q_b)),
// H = sum over the history lags of eta_d q+ - conj(eta_d) q-.  The part
// that does not depend on the history, exp(-(q_a-q_b)(eta_0 q_a - eta_0* q_b)),
// and the bare propagator U[a,a'] conj(U[b,b']) are folded into the table W.
// FP64: H splits into per-byte terms T_j of the representative's key, so
//   exp(-delta H) = prod_j exp(-delta T_j[byte_j]),
// read from tables of exp(-delta T) (no transcendental per group).
// C64: H is summed in FP32 with Kahan compensation over the per-byte terms
// (each stored as an FP32 hi + lo pair), then exp/sincos in FP32.
// History tables of one instance at one window length, in global or shared
// memory: FP32 hi/lo parts of the per-byte history terms, [chunk][256] each
// (C64 path), or exp(-delta_d T), [delta][chunk][256] (FP64 path).
struct Tab {
    const float2 *hi, *lo;
    const double2 *et;
};
__device__ __forceinline__ Tab tab_global(const Params &P, int n_act, int inst) {
    const size_t row = (size_t)(n_act - 1) * P.nchunks * kLutEntries;
    Tab t;
    t.hi = P.lutf + (size_t)inst * P.lut_stride + row;
    t.lo = P.lutf_lo + (size_t)inst * P.lut_stride + row;
    t.et = P.etab + (size_t)inst * P.etab_stride + (size_t)P.ndelta * row;
    return t;
}

// The end-point correction's tables (symmetric splitting) at a window length.
__device__ __forceinline__ Tab tab_E(const Params &P, int n_act) {
    const size_t row = (size_t)(n_act - 1) * P.nchunks * kLutEntries;
    Tab t;
    t.hi = P.lutEf + row;
    t.lo = P.lutElo + row;
    t.et = P.etabE + (size_t)P.ndelta * row;
    return t;
}

template <int M, bool C64>
struct Expander {
    static constexpr int MM = M * M;
    static constexpr int ND = M * (M - 1);   // at most this many distinct nonzero q_a - q_b
    using AmpT = typename std::conditional<C64, float2, double2>::type;

    template <typename T>
    static __device__ __forceinline__ T pick(const T *Ed, int d) {   // register select, no local memory
        T e = Ed[0];
#pragma unroll
        for (int i = 1; i < ND; ++i)
            if (i == d) e = Ed[i];
        return e;
    }

    // children of one group: v[k] amplitudes, returns the bit set of survivors
    // rho accumulators of one thread: FP64 on the FP64 path; on the C64 path
    // FP32 with a Kahan compensation term, widened to FP64 once per thread
    using AccT = typename std::conditional<C64, float2, double2>::type;

    static __device__ __forceinline__ void kahan_add(float2 &s, float2 &c, float2 a) {
        const float yx = a.x - c.x, tx = s.x + yx;
        c.x = (tx - s.x) - yx;
        s.x = tx;
        const float yy = a.y - c.y, ty = s.y + yy;
        c.y = (ty - s.y) - yy;
        s.y = ty;
    }

    // S: the group's merge sum (FP64), or on the C64 path already rounded to
    // FP32 (float2)
    template <typename SumT>
    static __device__ __forceinline__ unsigned children(const Params &P, int n_act, int inst, unsigned long long rep,
                                                        SumT S, const double2 *w, const float4 *wf, AmpT *v) {
        return children_tab(P, tab_global(P, n_act, inst), rep, S, w, wf, v);
    }

    // the same with the history tables given (tb: global or shared memory)
    template <typename SumT>
    static __device__ __forceinline__ unsigned children_tab(const Params &P, const Tab &tb, unsigned long long rep,
                                                            SumT S, const double2 *w, const float4 *wf, AmpT *v) {
        const unsigned c0 = (unsigned)(rep & ((1u << P.b) - 1u));
        const int pidx = (int)(c0 & ((1u << P.bs) - 1u)) * M + (int)(c0 >> P.bs);
        unsigned keep = 0;
        // Equally spaced coupling eigenvalues (q_a = q_0 + a s, P.qeq): the
        // difference of child (a, b) is (a - b) s, so its factor
        // exp(-(q_a - q_b) H) is E^(a-b) with E = exp(-s H) (or (1/E)^(b-a)):
        // one exponential and one sine/cosine per group, then products; which
        // power a child takes is fixed at compile time.  Otherwise one
        // factor per distinct difference, selected per child.
        const bool eq = P.qeq != 0;
        if constexpr (C64) {
            float2 Ed[ND];
            float2 Ep[M], En[M];   // Ep[n] = E^n, En[n] = E^-n (n >= 1)
            if (P.ndelta) {
                float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f, lx = 0.f, ly = 0.f;
                for (int j = 0; j < P.nchunks; ++j) {
                    const int idx = j * kLutEntries + (int)key_byte(rep, j);
                    const float2 hi = tb.hi[idx];
                    const float2 lo = tb.lo[idx];
                    const float yx = hi.x - cx, tx = sx + yx;
                    cx = (tx - sx) - yx;
                    sx = tx;
                    const float yy = hi.y - cy, ty = sy + yy;
                    cy = (ty - sy) - yy;
                    sy = ty;
                    lx += lo.x;
                    ly += lo.y;
                }
                const float hx = sx + (lx - cx), hy = sy + (ly - cy);
                if (eq) {
                    const float zr = -P.qstepf * hx, zi = -P.qstepf * hy;
                    float sn, cs;
                    sincosf(zi, &sn, &cs);
                    const float mp = expf(zr), mn = expf(-zr);
                    Ep[1] = make_float2(mp * cs, mp * sn);
                    En[1] = make_float2(mn * cs, -mn * sn);
#pragma unroll
                    for (int n = 2; n < M; ++n) {
                        Ep[n] = cmulf(Ep[n - 1], Ep[1]);
                        En[n] = cmulf(En[n - 1], En[1]);
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        if (d >= P.ndelta) break;
                        const float zr = -P.deltaf[d] * hx, zi = -P.deltaf[d] * hy;
                        float sn, cs;
                        sincosf(zi, &sn, &cs);
                        const float m = expf(zr);
                        Ed[d] = make_float2(m * cs, m * sn);
                    }
                }
            }
            const float2 Sf = to_f2(S);
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                // S (W_hi + W_lo): the table's FP32 rounding error is carried
                // (it would otherwise enter every step with the same sign and
                // add up over the trajectory); products of the small lo part
                // first, then fused into the hi products
                const float4 wv = wf[k * MM + pidx];
                const float lr = Sf.x * wv.z - Sf.y * wv.w, li = Sf.x * wv.w + Sf.y * wv.z;
                float2 a = make_float2(fmaf(Sf.x, wv.x, fmaf(-Sf.y, wv.y, lr)), fmaf(Sf.x, wv.y, fmaf(Sf.y, wv.x, li)));
                if (P.ndelta) {
                    if (eq) {
                        const int n = k / M - k % M;   // a - b
                        if (n > 0) a = cmulf(a, Ep[n]);
                        else if (n < 0) a = cmulf(a, En[-n]);
                    } else {
                        const int d = P.dsel[k];
                        if (d >= 0) a = cmulf(a, pick(Ed, d));
                    }
                }
                v[k] = a;
                if (a.x * a.x + a.y * a.y >= P.theta2f) keep |= 1u << k;
            }
        } else {
            double2 Ed[ND];
            double2 Ep[M], En[M];
            const int dstride = P.nchunks * kLutEntries;
            if (eq && P.ndelta) {
                double2 ep = make_double2(1.0, 0.0), en = make_double2(1.0, 0.0);
                for (int j = 0; j < P.nchunks; ++j) {
                    const int idx = j * kLutEntries + (int)key_byte(rep, j);
                    ep = cmul(ep, tb.et[P.d_pos * dstride + idx]);
                    en = cmul(en, tb.et[P.d_neg * dstride + idx]);
                }
                Ep[1] = ep;
                En[1] = en;
#pragma unroll
                for (int n = 2; n < M; ++n) {
                    Ep[n] = cmul(Ep[n - 1], ep);
                    En[n] = cmul(En[n - 1], en);
                }
            } else {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    if (d >= P.ndelta) break;
                    double2 e = make_double2(1.0, 0.0);
                    for (int j = 0; j < P.nchunks; ++j) e = cmul(e, tb.et[d * dstride + j * kLutEntries + (int)key_byte(rep, j)]);
                    Ed[d] = e;
                }
            }
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                double2 a = cmul(S, w[k * MM + pidx]);
                if (P.ndelta) {
                    if (eq) {
                        const int n = k / M - k % M;
                        if (n > 0) a = cmul(a, Ep[n]);
                        else if (n < 0) a = cmul(a, En[-n]);
                    } else {
                        const int d = P.dsel[k];
                        if (d >= 0) a = cmul(a, pick(Ed, d));
                    }
                }
                v[k] = a;
                if (a.x * a.x + a.y * a.y >= P.theta2) keep |= 1u << k;
            }
        }
        return keep;
    }
};

// Block partial of the threads' rho accumulators into out[0 .. MM): per
// component the thread's value is hi + lo.  C64 (FP32 sum and compensation):
// each warp reduces with error-free additions (TwoSum, every rounding error
// carried into the lo part) and widens to FP64 once, in lane 0, so that the
// reduction stays off the FP64 pipe (1/64 of the FP32 rate on this part);
// FP64 accumulators (lo unused) reduce with FP64 shuffles.  Warps are summed
// in FP64, in warp order.  s_r: [NW][MM] scratch; every thread of the block
// calls it.
template <int MM, int NW, bool C64>
__device__ __forceinline__ void block_rho_partial(const typename std::conditional<C64, float2, double2>::type *hi,
                                                  const float2 *lo, double2 (*s_r)[MM], double2 *out) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MM; ++k) {
        if constexpr (C64) {
            float sx = hi[k].x, ex = lo[k].x, sy = hi[k].y, ey = lo[k].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float bx = __shfl_down_sync(0xffffffffu, sx, o), fx = __shfl_down_sync(0xffffffffu, ex, o);
                const float by = __shfl_down_sync(0xffffffffu, sy, o), fy = __shfl_down_sync(0xffffffffu, ey, o);
                const float tx = sx + bx, vx = tx - sx;
                ex += fx + ((sx - (tx - vx)) + (bx - vx));
                sx = tx;
                const float ty = sy + by, vy = ty - sy;
                ey += fy + ((sy - (ty - vy)) + (by - vy));
                sy = ty;
            }
            if (lane == 0) s_r[warp][k] = make_double2(f2d_exact(sx) + f2d_exact(ex), f2d_exact(sy) + f2d_exact(ey));
        } else {
            double x = hi[k].x, y = hi[k].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_down_sync(0xffffffffu, x, o);
                y += __shfl_down_sync(0xffffffffu, y, o);
            }
            if (lane == 0) s_r[warp][k] = make_double2(x, y);
        }
    }
    __syncthreads();
    if (threadIdx.x < MM) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < NW; ++w) {
            x += s_r[w][threadIdx.x].x;
            y += s_r[w][threadIdx.x].y;
        }
        out[threadIdx.x] = make_double2(x, y);
    }
}

// Extension of n groups (merge steps) or n stored paths (while the window
// fills) to their children; survivors appended through *cnt_out.  This
// block's partial sums of rho(t+1) (and its survivor count) per instance go
// to part[blockIdx.x][inst][0 .. M*M].  Single problems accumulate in
// registers (FP64, or FP32 + Kahan on the C64 path); batches accumulate per
// instance in shared memory (FP64 atomics; dynamic shared memory of
// n_inst * (M*M + 1) double2).
template <int M, bool C64, int NT, bool BATCH>
__device__ __forceinline__ void phase_expand(const Params &P, unsigned long long t, unsigned long long n, bool merge,
                                             unsigned long long *cnt_out, double2 *part,
                                             unsigned long long *keys_dst = nullptr, void *amps_dst = nullptr) {
    using X = Expander<M, C64>;
    using AmpT = typename X::AmpT;
    constexpr int MM = M * M;
    constexpr int NW = NT / 32;
    DevState *st = P.st;
    const unsigned long long tn = t + 1;
    const int n_act = (int)min(tn, (unsigned long long)P.dkmax);
    const int L_child = (int)min(tn + 1, (unsigned long long)P.dkmax);
    const unsigned long long wmask = (P.b * L_child >= 64) ? ~0ull : ((1ull << (P.b * L_child)) - 1ull);
    const unsigned long long *keys_in = P.keys[t & 1];
    const AmpT *amps_in = static_cast<const AmpT *>(P.amps[t & 1]);
    // survivors go to the other ping-pong buffer, or where the caller says
    // (the post-merging engine's unmerged buffer)
    unsigned long long *keys_out = keys_dst ? keys_dst : P.keys[tn & 1];
    AmpT *amps_out = static_cast<AmpT *>(amps_dst ? amps_dst : P.amps[tn & 1]);

    __shared__ double2 s_w[MM * MM];
    __shared__ float4 s_wf[MM * MM];
    __shared__ double2 s_r[NW][MM];
    extern __shared__ double2 s_acc[];   // BATCH: [n_inst][MM + 1]
    if constexpr (BATCH) {
        for (int i = threadIdx.x; i < P.n_inst * (MM + 1); i += NT) s_acc[i] = make_double2(0.0, 0.0);
    } else {
        for (int i = threadIdx.x; i < MM * MM; i += NT) {
            s_w[i] = P.wtab[i];
            s_wf[i] = P.wtabf[i];
        }
    }
    __syncthreads();

    typename X::AccT racc[BATCH ? 1 : MM], rcmp[BATCH ? 1 : MM];
#pragma unroll
    for (int k = 0; k < (BATCH ? 1 : MM); ++k) {
        racc[k].x = racc[k].y = 0;
        rcmp[k].x = rcmp[k].y = 0;
    }
    unsigned long long block_kept = 0;

    const unsigned long long stride = (unsigned long long)gridDim.x * NT;
    for (unsigned long long base = blockIdx.x * (unsigned long long)NT; base < n; base += stride) {
        const unsigned long long g = base + threadIdx.x;
        unsigned keepbits = 0;
        AmpT camp[MM];
        unsigned long long rep = 0;
        int inst = 0;
        if (g < n) {
            double2 S;
            if (merge) {
                const unsigned int h = __ldcg(P.groups + g);
                rep = __ldcg(P.repk + h);
                S = __ldcg(reinterpret_cast<const double2 *>(&P.slots[h].sre));
                Slot fresh;
                fresh.mk = kEmpty;
                fresh.wmax = 0ull;
                fresh.sre = 0.0;
                fresh.sim = 0.0;
                P.slots[h] = fresh;
                P.repk[h] = kEmpty;
            } else {
                rep = __ldcg(keys_in + g);
                S = load_amp(amps_in, g);
            }
            if constexpr (BATCH) {
                inst = (int)(rep >> P.inst_shift);
                keepbits = X::children(P, n_act, inst, rep, S, P.wtab + (size_t)inst * MM * MM,
                                       P.wtabf + (size_t)inst * MM * MM, camp);
                double2 *acc = s_acc + (size_t)inst * (MM + 1);
#pragma unroll
                for (int k = 0; k < MM; ++k)
                    if (keepbits & (1u << k)) {
                        atomicAdd(&acc[k].x, (double)camp[k].x);
                        atomicAdd(&acc[k].y, (double)camp[k].y);
                    }
                if (keepbits) atomicAdd(&acc[MM].x, (double)__popc(keepbits));
            } else {
                keepbits = X::children(P, n_act, 0, rep, S, s_w, s_wf, camp);
                if (P.sym) {
                    // symmetric splitting: rho(t) takes every surviving child
                    // times its newest point's end-point correction (the
                    // stored child keeps the interior factors)
                    AmpT cr[MM];
                    X::children_tab(P, tab_E(P, n_act), rep, make_double2(1.0, 0.0), P.wEt, P.wEtf, cr);
#pragma unroll
                    for (int k = 0; k < MM; ++k)
                        if (keepbits & (1u << k)) {
                            if constexpr (C64) {
                                X::kahan_add(racc[k], rcmp[k], cmulf(camp[k], cr[k]));
                            } else {
                                const double2 v = cmul(camp[k], cr[k]);
                                racc[k].x += v.x;
                                racc[k].y += v.y;
                            }
                        }
                } else {
#pragma unroll
                    for (int k = 0; k < MM; ++k)
                        if (keepbits & (1u << k)) {
                            if constexpr (C64) {
                                X::kahan_add(racc[k], rcmp[k], camp[k]);
                            } else {
                                racc[k].x += camp[k].x;
                                racc[k].y += camp[k].y;
                            }
                        }
                }
            }
        }
        const unsigned cnt = __popc(keepbits);
        const Append ap = block_append<NT>(cnt, cnt_out);
        block_kept += ap.total;
        if (ap.total && ap.base + ap.total > (unsigned long long)P.max_paths) {
            if (threadIdx.x == 0) raise_err(st, kErrPaths);
        } else if (cnt) {
            unsigned long long o = ap.base + ap.excl;
            const unsigned long long shifted = rep << P.b;
            const unsigned long long ibits = rep & P.instmask;
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                if (keepbits & (1u << k)) {
                    const unsigned long long code = (unsigned long long)((k / M) | ((k % M) << P.bs));
                    keys_out[o] = ((shifted | code) & wmask) | ibits;
                    amps_out[o] = camp[k];
                    ++o;
                }
            }
        }
    }
    double2 *mine = part + (size_t)blockIdx.x * P.n_inst * (MM + 1);
    if constexpr (BATCH) {
        __syncthreads();
        for (int i = threadIdx.x; i < P.n_inst * (MM + 1); i += NT) mine[i] = s_acc[i];
    } else {
        // this block's partial sums
        float2 lo[MM];
#pragma unroll
        for (int k = 0; k < MM; ++k) {
            if constexpr (C64) lo[k] = make_float2(-rcmp[k].x, -rcmp[k].y);
            else lo[k] = make_float2(0.f, 0.f);
        }
        block_rho_partial<MM, NW, C64>(racc, lo, s_r, mine);
        if (threadIdx.x == 0) mine[MM] = make_double2((double)block_kept, 0.0);
    }
    __syncthreads();
}

// One block, one instance: rho(tn) of the instance and its survivor count
// from the nblk per-block partials, summed in block order (deterministic).
__device__ __forceinline__ void phase_finalize(const Params &P, unsigned long long tn, int inst, const double2 *part,
                                               int nblk, int MM) {
    __shared__ double2 s_p[256];
    const int MM1 = MM + 1;
    const size_t pstride = (size_t)P.n_inst * MM1;
    const double2 *src = part + (size_t)inst * MM1;
    // T threads per element k sum a fixed stride of the partials; each
    // round issues all of a thread's (up to 8) loads before adding, so that
    // up to 8T partials per element cost one trip to L2
    const int T = min((int)blockDim.x, 256) / MM1;
    const int k = (int)threadIdx.x / T, sidx = (int)threadIdx.x % T;
    double2 a = make_double2(0.0, 0.0);
    if (k < MM1 && threadIdx.x < 256) {
        for (int b0 = sidx; b0 < nblk; b0 += 8 * T) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int b = b0 + u * T;
                v[u] = b < nblk ? __ldcg(src + (size_t)b * pstride + k) : make_double2(0.0, 0.0);
            }
            a.x += ((v[0].x + v[1].x) + (v[2].x + v[3].x)) + ((v[4].x + v[5].x) + (v[6].x + v[7].x));
            a.y += ((v[0].y + v[1].y) + (v[2].y + v[3].y)) + ((v[4].y + v[5].y) + (v[6].y + v[7].y));
        }
    }
    if (threadIdx.x < 256) s_p[threadIdx.x] = a;
    __syncthreads();
    // the T partials of element k: pairwise tree in shared memory
    for (int w = 1; w < T; w <<= 1) {
        if (k < MM1 && threadIdx.x < 256 && (sidx % (2 * w)) == 0 && sidx + w < T) {
            s_p[threadIdx.x].x += s_p[threadIdx.x + w].x;
            s_p[threadIdx.x].y += s_p[threadIdx.x + w].y;
        }
        __syncthreads();
    }
    if ((int)threadIdx.x < MM1) {
        const double x = s_p[threadIdx.x * T].x, y = s_p[threadIdx.x * T].y;
        const size_t slot = (size_t)(tn % (unsigned long long)P.rho_hist);
        if ((int)threadIdx.x < MM)
            P.rho_ring[(slot * P.n_inst + inst) * MM + threadIdx.x] = make_double2(x, y);
        else
            P.inst_kept[slot * P.n_inst + inst] = (long long)(x + 0.5);
    }
    __syncthreads();
}

__device__ __forceinline__ void write_step_totals(const Params &P, unsigned long long tn, unsigned long long groups,
                                                  unsigned long long n_out, int MM) {
    StepRec r;
    r.t = (long long)tn;
    r.groups = (long long)groups;
    r.extended = (long long)groups * MM;
    r.kept = (long long)n_out;
    r.inter = (long long)n_out;   // pre-merging: the largest set of the step is the stored one
    P.stats_ring[tn % (unsigned long long)P.rho_hist] = r;
}

struct StepCounts {
    unsigned long long groups, n_out;
};
// The step's counters (read through L2: other blocks of the same kernel
// wrote them); the last block reads them while it sums the partials.
__device__ __forceinline__ StepCounts step_counts(const Params &P, DevState *st, unsigned long long tn) {
    const bool merge = tn >= (unsigned long long)P.dkmax;
    StepCounts c;
    c.groups = merge ? __ldcg(&st->cnt_groups[tn % 3]) : __ldcg(&st->n_cur);
    c.n_out = __ldcg(&st->cnt_out[tn % 3]);
    return c;
}
// Publishes step tn (one thread, after every block of the step is done):
// totals, the new count and time, and zeroed counters of the next step.
__device__ __forceinline__ void publish_step(const Params &P, DevState *st, unsigned long long tn, int MM,
                                             StepCounts c) {
    *P.fin_count = 0;
    const unsigned long long groups = c.groups, n_out = c.n_out;
    write_step_totals(P, tn, groups, n_out, MM);
    st->n_cur = n_out;
    st->t = tn;
    st->cnt_groups[(tn + 1) % 3] = 0;   // counters of the next step
    st->cnt_out[(tn + 1) % 3] = 0;
    st->ticket[(tn + 1) % 3] = 0;
}

__device__ __forceinline__ double2 *rho_part_of(const Params &P, unsigned long long tn, int MM) {
    return P.rho_part + (size_t)(tn & 1) * kMaxExpandBlocks * P.n_inst * (MM + 1);
}

// Stream engine: each block stores its partial of rho per end point, C64 as
// an FP32 sum and the rounding error of every addition (warp shuffles, then
// the warps folded by one thread per end point, all with error-free TwoSum
// additions, so no FP64 in the kernel's tail), FP64 as a double pair in the
// same 16 bytes.  s_rt: [NW][M*M] scratch; dst = [M*M] of this block.  All
// threads of the block call it.
template <int MM, int NW, bool C64>
__device__ __forceinline__ void block_rho_pair(const typename std::conditional<C64, float2, double2>::type *hi,
                                               const float2 *lo, float4 (*s_rt)[MM], float4 *dst) {
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MM; ++k) {
        if constexpr (C64) {
            float sx = hi[k].x, ex = lo[k].x, sy = hi[k].y, ey = lo[k].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float bx = __shfl_down_sync(0xffffffffu, sx, o), fx = __shfl_down_sync(0xffffffffu, ex, o);
                const float by = __shfl_down_sync(0xffffffffu, sy, o), fy = __shfl_down_sync(0xffffffffu, ey, o);
                const float tx = sx + bx, vx = tx - sx;
                ex += fx + ((sx - (tx - vx)) + (bx - vx));
                sx = tx;
                const float ty = sy + by, vy = ty - sy;
                ey += fy + ((sy - (ty - vy)) + (by - vy));
                sy = ty;
            }
            if (lane == 0) s_rt[warp][k] = make_float4(sx, ex, sy, ey);
        } else {
            double x = hi[k].x, y = hi[k].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_down_sync(0xffffffffu, x, o);
                y += __shfl_down_sync(0xffffffffu, y, o);
            }
            if (lane == 0) reinterpret_cast<double2 *>(&s_rt[warp][0])[k] = make_double2(x, y);
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < MM) {
        const int k = threadIdx.x;
        if constexpr (C64) {
            float4 a = s_rt[0][k];
            for (int w = 1; w < NW; ++w) {
                const float4 b = s_rt[w][k];
                const float tx = a.x + b.x, vx = tx - a.x;
                a.y += b.y + ((a.x - (tx - vx)) + (b.x - vx));
                a.x = tx;
                const float ty = a.z + b.z, vy = ty - a.z;
                a.w += b.w + ((a.z - (ty - vy)) + (b.z - vy));
                a.z = ty;
            }
            dst[k] = a;
        } else {
            double2 a = reinterpret_cast<const double2 *>(&s_rt[0][0])[k];
            for (int w = 1; w < NW; ++w) {
                const double2 b = reinterpret_cast<const double2 *>(&s_rt[w][0])[k];
                a.x += b.x;
                a.y += b.y;
            }
            reinterpret_cast<double2 *>(dst)[k] = a;
        }
    }
}

__device__ __forceinline__ float4 *spart_of(const Params &P, unsigned long long tn, int MM) {
    return P.spart + (size_t)(tn & 1) * kMaxExpandBlocks * MM;
}
__device__ __forceinline__ long long *scount_of(const Params &P, unsigned long long tn) {
    return P.scount + (size_t)(tn & 1) * kMaxExpandBlocks;
}

// rho(tn) of the stream engine from the per-block partials of nblk blocks,
// summed in a fixed order, and the survivor count.  Block-uniform (a
// multiple of 32 threads, at most 1024).
template <bool C64>
__device__ __forceinline__ void phase_finalize_stream(const Params &P, unsigned long long tn, int nblk, int MM) {
    // one warp per component (re, im of each end point): lane l adds the
    // partials of blocks l, l + 32, ... in order, then a shuffle tree.  C64
    // partials are FP32 pairs: lanes add them with TwoSum and the warp merges
    // the pairs error-free, so FP64 is used once per component; FP64 pairs
    // are added in FP64.  Counts: per-thread sums, then a shuffle tree and the
    // warps in order.
    __shared__ double s_p[64];
    __shared__ long long s_c[32];
    const float4 *src = spart_of(P, tn, MM);
    const long long *cnt = scount_of(P, tn);
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int comp = (int)warp; comp < 2 * MM; comp += (int)nw) {
        const int k = comp >> 1, im = comp & 1;
        if constexpr (C64) {
            float sh = 0.f, se = 0.f;
#pragma unroll 4
            for (int w = (int)lane; w < nblk; w += 32) {
                const float4 q = __ldcg(src + (size_t)w * MM + k);
                two_sum_acc(sh, se, im ? q.z : q.x);
                se += im ? q.w : q.y;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float b = __shfl_down_sync(0xffffffffu, sh, o), f = __shfl_down_sync(0xffffffffu, se, o);
                const float t = sh + b, v = t - sh;
                se += f + ((sh - (t - v)) + (b - v));
                sh = t;
            }
            if (lane == 0) s_p[comp] = f2d_exact(sh) + f2d_exact(se);
        } else {
            double a = 0.0;
#pragma unroll 4
            for (int w = (int)lane; w < nblk; w += 32) {
                const float4 q = __ldcg(src + (size_t)w * MM + k);
                const double2 d = *reinterpret_cast<const double2 *>(&q);
                a += im ? d.y : d.x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) s_p[comp] = a;
        }
    }
    long long c = 0;
    for (int b = (int)threadIdx.x; b < nblk; b += (int)blockDim.x) c += __ldcg(cnt + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) s_c[warp] = c;
    __syncthreads();
    const size_t slot = (size_t)(tn % (unsigned long long)P.rho_hist);
    if ((int)threadIdx.x < MM)
        P.rho_ring[slot * MM + threadIdx.x] = make_double2(s_p[2 * threadIdx.x], s_p[2 * threadIdx.x + 1]);
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (unsigned w = 0; w < nw; ++w) tot += s_c[w];
        P.inst_kept[slot] = tot;
    }
    __syncthreads();
}

// The stream kernels' last block publishes a step's counters and leaves the
// sum of the blocks' partials of rho to block 0 of the next step (or to
// k_rho_finalize before a read): rho(t) of a step is complete when the next
// step starts or the host reads it.  Partials alternate by step parity, so
// the next step's own partials never overwrite them.  Block-uniform.
template <bool C64>
__device__ __forceinline__ void finish_pending_rho(const Params &P, DevState *st, int MM) {
    const unsigned long long pt = st->rho_pending;
    if (pt == 0) return;
    phase_finalize_stream<C64>(P, pt, (int)st->rho_nblk, MM);
    if (threadIdx.x == 0) st->rho_pending = 0;
}

// Batches of the stream engine: rho(t) and the survivor count of the
// pending step per instance, instance i by block i (then i + gridDim.x, ...),
// from the blocks' partials ([block][instance][M*M + 1], phase_finalize:
// summed in block order).  The step kernels leave the mark (each block
// reads it; the next step's last block replaces it); a one-block read-time
// call clears it.  Block-uniform.
__device__ __forceinline__ void finish_pending_rho_batch(const Params &P, DevState *st, int MM, bool clear) {
    const unsigned long long pt = __ldcg(&st->rho_pending);
    if (pt == 0) return;
    const int nblk = (int)__ldcg(&st->rho_nblk);
    for (int inst = blockIdx.x; inst < P.n_inst; inst += gridDim.x)
        phase_finalize(P, pt, inst, rho_part_of(P, pt, MM), nblk, MM);
    if (clear && threadIdx.x == 0) st->rho_pending = 0;
}

template <bool C64>
__global__ void k_rho_finalize(Params P, int MM) {
    if (P.st->err) return;
    if (P.n_inst > 1) finish_pending_rho_batch(P, P.st, MM, gridDim.x == 1);
    else finish_pending_rho<C64>(P, P.st, MM);
}

// The same (finalize: stream engine), then rho(t0 ...) for nelem = count *
// n_inst * M*M entries written to dst, host memory the device can address
// (page-locked): no separate copy.  One block.
template <bool C64>
__global__ void k_rho_read_to(Params P, int MM, int finalize, double2 *dst, long long t0, long long nelem) {
    if (finalize && !P.st->err) {
        if (P.n_inst > 1) finish_pending_rho_batch(P, P.st, MM, true);
        else finish_pending_rho<C64>(P, P.st, MM);
    }
    const long long per = (long long)P.n_inst * MM;
    for (long long i = threadIdx.x; i < nelem; i += blockDim.x) {
        const long long t = t0 + i / per;
        dst[i] = P.rho_ring[(size_t)(t % P.rho_hist) * per + i % per];
    }
}

template <int M, bool C64, bool BATCH>
__global__ void __launch_bounds__(kExpandThreads) k_expand(Params P) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    const bool merge = tn >= (unsigned long long)P.dkmax;
    const unsigned long long n = merge ? st->cnt_groups[tn % 3] : st->n_cur;
    phase_expand<M, C64, kExpandThreads, BATCH>(P, t, n, merge, &st->cnt_out[tn % 3], rho_part_of(P, tn, M * M));
}

// Step finalisation of the multi-kernel path: block i finalises instance i;
// the last block to finish publishes the step (counts, t, next counters).
__global__ void __launch_bounds__(256) k_finalize(Params P, int MM, int nblk) {
    DevState *st = P.st;
    __shared__ bool s_last;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    for (int inst = blockIdx.x; inst < P.n_inst; inst += gridDim.x)
        phase_finalize(P, tn, inst, rho_part_of(P, tn, MM), nblk, MM);
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(P.fin_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    publish_step(P, st, tn, MM, step_counts(P, st, tn));
}

// Grid-wide barrier of the persistent kernel (all blocks are co-resident: the
// kernel is launched cooperatively).  The wait is bounded: after
// kBarrierCycles, or as soon as another block has raised an error, the block
// stops waiting and the timeout is recorded.  Returns the error bits.
__device__ __forceinline__ unsigned grid_barrier(DevState *st) {
    __shared__ unsigned s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &st->bar_gen;
        volatile unsigned *verr = &st->err;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&st->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            st->bar_count = 0;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (*verr) break;
                if (clock64() - t0 > kBarrierCycles) {
                    atomicOr(&st->err, kErrTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_err = *verr;
    }
    __syncthreads();
    return s_err;
}

// All steps of one qp_step call in one cooperative launch.  Per step: insert
// | tiebreak | expand, separated by grid barriers (only expand while the
// window fills).  Step t' is finalised at the start of step t'+1 (and the
// last step after the loop) from values every block already holds: block b
// finalises instances b, b + gridDim.x, ...; block 0 writes the totals.
// Counter sets rotate mod 3 so that no counter is reset while a block may
// still read it.
template <int M, bool C64, bool BATCH>
__global__ void __launch_bounds__(kPersistThreads) k_step_persistent(Params P, int nsteps) {
    constexpr int MM = M * M;
    using Amp = typename Expander<M, C64>::AmpT;
    DevState *st = P.st;
    const int nblk = (int)gridDim.x;
    unsigned err = *(volatile unsigned *)&st->err;
    unsigned long long t = st->t;
    unsigned long long n_in = st->n_cur;
    unsigned long long prev_groups = 0, prev_out = 0;
    int done = 0;
    for (int s = 0; s < nsteps && !err; ++s) {
        const unsigned long long tn = t + 1;
        const int cs = (int)(tn % 3);
        const bool merge = tn >= (unsigned long long)P.dkmax;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            st->cnt_groups[(tn + 1) % 3] = 0;   // last used two steps ago
            st->cnt_out[(tn + 1) % 3] = 0;
            if (s > 0) write_step_totals(P, t, prev_groups, prev_out, MM);
        }
        if (s > 0)
            for (int inst = blockIdx.x; inst < P.n_inst; inst += nblk)
                phase_finalize(P, t, inst, rho_part_of(P, t, MM), nblk, MM);
        if (merge) {
            phase_insert<Amp, kPersistThreads>(P, t, n_in, &st->cnt_groups[cs]);
            err = grid_barrier(st);
            if (err) break;
            phase_tiebreak<Amp, kPersistThreads>(P, t, n_in);
            err = grid_barrier(st);
            if (err) break;
        }
        const unsigned long long ng = merge ? __ldcg(&st->cnt_groups[cs]) : n_in;
        phase_expand<M, C64, kPersistThreads, BATCH>(P, t, ng, merge, &st->cnt_out[cs], rho_part_of(P, tn, MM));
        err = grid_barrier(st);
        if (err) break;
        prev_groups = ng;
        prev_out = __ldcg(&st->cnt_out[cs]);
        n_in = prev_out;
        t = tn;
        ++done;
    }
    if (done > 0) {
        for (int inst = blockIdx.x; inst < P.n_inst; inst += nblk)
            phase_finalize(P, t, inst, rho_part_of(P, t, MM), nblk, MM);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            write_step_totals(P, t, prev_groups, prev_out, MM);
            st->n_cur = n_in;
            st->t = t;
        }
    }
}

// ---------------------------------------------------------------- stream engine

// Look-back word: (step epoch << 32) | (state << 30) | count.
__device__ __forceinline__ unsigned long long lb_word(unsigned epoch, unsigned state, unsigned long long cnt) {
    return ((unsigned long long)epoch << 32) | ((unsigned long long)state << 30) | cnt;
}

// Regular steps of the stream engine (no filter, see Params): while the
// window fills every stored path is its own group; with the full mask, once
// all M^(2 dkmax) keys are stored, every group is the M*M consecutive values
// of the oldest point.  Every child survives, so child c of group g goes to
// entry g of output region c: a streaming map, one thread per group, no
// shared-memory tile, no look-back.  The representative does not
// matter: members differ only in the oldest point, which the history sum
// does not read and the child key drops.  Launched before the tile kernel on
// configurations that allow regular steps; it decides on the device, takes
// the step (reg_done = new t + 1) or leaves it to the tile kernel
// (reg_done = 0), and publishes the step it takes like the tile kernel.
template <int M, bool C64>
__global__ void __launch_bounds__(kRegThreads, 3) k_stream_regular(Params P, int lut_smem) {
    using X = Expander<M, C64>;
    using AmpT = typename X::AmpT;
    constexpr int MM = M * M, NT = kRegThreads;
    static_assert(NT / 32 == kStreamWarps, "warp partials");
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    const int in = (int)(t & 1), outp = (int)(tn & 1), cs = (int)(tn % 3);
    const bool merge = tn >= (unsigned long long)P.dkmax;
    const long long G = P.region_cap;
    __shared__ long long s_gb[MM + 1];
    __shared__ double2 s_w[C64 ? 1 : MM * MM];
    __shared__ float4 s_wf[MM * MM];
    __shared__ float4 s_rt[kRegThreads / 32][MM];
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        long long acc = 0;
        const int gsz = merge ? MM : 1;
        unsigned long long n_in = 0;
        for (int r = 0; r < MM; ++r) {
            const long long nr = (long long)__ldcg(&P.reg_n[in * MM + r]);
            n_in += (unsigned long long)nr;
            s_gb[r] = acc;
            acc += nr / gsz;
        }
        const bool regular = n_in > 0 && (merge ? (P.reg_merge && n_in == P.full_n) : (P.reg_fill != 0));
        s_gb[MM] = regular ? acc : -1;
    }
    __syncthreads();
    const long long ngroups = s_gb[MM];
    if (ngroups < 0) {   // not a regular step: the tile kernel takes it
        if (blockIdx.x == 0 && threadIdx.x == 0) st->reg_done = 0;
        return;
    }
    if (blockIdx.x == 0) finish_pending_rho<C64>(P, st, MM);   // rho of the previous step
    const int gs = merge ? MM : 1;
    const int n_act = (int)min(tn, (unsigned long long)P.dkmax);
    const int L_child = (int)min(tn + 1, (unsigned long long)P.dkmax);
    const unsigned long long wmask = (P.b * L_child >= 64) ? ~0ull : ((1ull << (P.b * L_child)) - 1ull);
    const unsigned long long *keys_in = P.keys[in];
    const AmpT *amps_in = static_cast<const AmpT *>(P.amps[in]);
    unsigned long long *keys_out = P.keys[outp];
    AmpT *amps_out = static_cast<AmpT *>(P.amps[outp]);
    extern __shared__ __align__(16) unsigned char s_dyn[];
    for (int i = threadIdx.x; i < MM * MM; i += NT) {
        if constexpr (!C64) s_w[i] = P.wtab[i];
        s_wf[i] = P.wtabf[i];
    }
    Tab tab = tab_global(P, n_act, 0);
    if (lut_smem && P.ndelta) {
        const int n = P.nchunks * kLutEntries;
        if constexpr (C64) {
            float2 *hi = reinterpret_cast<float2 *>(s_dyn), *lo = hi + n;
            for (int i = threadIdx.x; i < n; i += NT) {
                hi[i] = __ldg(tab.hi + i);
                lo[i] = __ldg(tab.lo + i);
            }
            tab.hi = hi;
            tab.lo = lo;
        } else {
            double2 *et = reinterpret_cast<double2 *>(s_dyn);
            for (int i = threadIdx.x; i < n * P.ndelta; i += NT) et[i] = __ldg(tab.et + i);
            tab.et = et;
        }
    }
    if (blockIdx.x == 0) {
        if ((int)threadIdx.x < MM) P.reg_n[outp * MM + threadIdx.x] = (unsigned long long)ngroups;
        if (threadIdx.x == 0) {
            st->cnt_out[cs] = (unsigned long long)ngroups * MM;
            st->cnt_groups[cs] = (unsigned long long)ngroups;
            st->reg_done = tn + 1;
        }
    }
    __syncthreads();
    constexpr bool kKahan = C64;
    typename X::AccT racc[MM], rcmp[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) {
        racc[k].x = racc[k].y = 0;
        rcmp[k].x = rcmp[k].y = 0;
    }
    // a group's members: vector loads (a group of M*M entries starts on a
    // multiple of M*M of a region whose base is 16-entry aligned)
    struct Members {
        unsigned long long rk;
        AmpT a[MM];
    };
    auto load = [&](long long g, Members &mb) {
        int r = 0;
        while (r + 1 < MM && g >= s_gb[r + 1]) ++r;
        const long long j = (g - s_gb[r]) * gs;
        mb.rk = __ldcs(keys_in + r * G + j);
        if (gs == 1) {
            mb.a[0] = __ldcs(amps_in + r * G + j);
        } else if constexpr (C64 && MM % 2 == 0) {
            const float4 *p4 = reinterpret_cast<const float4 *>(amps_in + r * G + j);
#pragma unroll
            for (int m = 0; m < MM / 2; ++m) {
                const float4 q = __ldcs(p4 + m);
                mb.a[2 * m] = make_float2(q.x, q.y);
                mb.a[2 * m + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int m = 0; m < MM; ++m) mb.a[m] = __ldcs(amps_in + r * G + j + m);
        }
    };
    // one group: sum (C64: FP32 with every rounding error kept, TwoSum, in
    // member order and rounded once, as the tile kernel's owner threads do;
    // FP64: FP64), children, write, accumulate rho
    auto group = [&](long long g, const Members &mb) {
        const unsigned long long rk = mb.rk;
        AmpT v[MM];
        if (gs == 1) {   // a single member is its own sum, exactly
            X::children_tab(P, tab, rk, mb.a[0], s_w, s_wf, v);
        } else if constexpr (C64) {
            float sx = mb.a[0].x, sy = mb.a[0].y, ex = 0.f, ey = 0.f;
#pragma unroll
            for (int m = 1; m < MM; ++m) {
                two_sum_acc(sx, ex, mb.a[m].x);
                two_sum_acc(sy, ey, mb.a[m].y);
            }
            X::children_tab(P, tab, rk, make_float2(sx + ex, sy + ey), s_w, s_wf, v);
        } else {
            double sx = mb.a[0].x, sy = mb.a[0].y;
#pragma unroll
            for (int m = 1; m < MM; ++m) {
                sx += mb.a[m].x;
                sy += mb.a[m].y;
            }
            X::children_tab(P, tab, rk, make_double2(sx, sy), s_w, s_wf, v);
        }
        const unsigned long long shifted = rk << P.b;
#pragma unroll
        for (int c = 0; c < MM; ++c) {
            const unsigned long long code = (unsigned long long)((c / M) | ((c % M) << P.bs));
            keys_out[c * G + g] = (shifted | code) & wmask;
            amps_out[c * G + g] = v[c];
            if constexpr (kKahan) {
                X::kahan_add(racc[c], rcmp[c], v[c]);
            } else {
                racc[c].x += v[c].x;
                racc[c].y += v[c].y;
            }
        }
    };
    const long long stride = (long long)gridDim.x * NT;
    if (ngroups > G) {   // the outputs would not fit their regions
        if (threadIdx.x == 0) raise_err(st, kErrPaths);
    } else {
        // one group per thread at a time: three blocks of eight warps per SM
        // keep more bytes in flight than two groups per thread at two blocks
        for (long long g = (long long)blockIdx.x * NT + threadIdx.x; g < ngroups; g += stride) {
            Members m0;
            load(g, m0);
            group(g, m0);
        }
    }
    // arrive first: the last block to arrive publishes the step, for which
    // it needs the step's counters only; every block then writes its partial
    // of rho, which the next step's block 0 (or a read-time finalisation)
    // sums once this kernel has ended
    __syncthreads();
    if (threadIdx.x == 0) {
        // one acquire-release add: releases this block's writes (ordered
        // before it by the barrier), and the last block acquires the others'
        s_last = atom_add_acq_rel_gpu(P.fin_count, 1u) == gridDim.x - 1;
        if (s_last) {
            if (__ldcg(&st->err)) {   // a failed step is not published
                *P.fin_count = 0;
            } else {
                st->rho_nblk = gridDim.x;
                st->rho_pending = tn;
                publish_step(P, st, tn, MM, step_counts(P, st, tn));
            }
        }
    }
    // block partials of rho(tn) and the children written by this block
    float4 *mine = spart_of(P, tn, MM) + (size_t)blockIdx.x * MM;
    float2 lo[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) lo[k] = C64 ? make_float2(-(float)rcmp[k].x, -(float)rcmp[k].y) : make_float2(0.f, 0.f);
    block_rho_pair<MM, kRegThreads / 32, C64>(racc, lo, s_rt, mine);
    if (threadIdx.x == 0) {
        long long mg = 0;
        for (long long g0 = (long long)blockIdx.x * NT; g0 < ngroups; g0 += stride) mg += min((long long)NT, ngroups - g0);
        scount_of(P, tn)[blockIdx.x] = mg * MM;
    }
}

// The groups of runs of at most this many stored paths are summed by one
// owner thread each (stream engine); longer runs, which occur only while the
// window fills, by shared FP64 atomics.
constexpr int kOwnRun = 32;
// A group sum formed in FP32 by its run's thread is stored as the float2 in
// the low 8 bytes of its double2 slot and this signalling-NaN pattern in the
// high 8 (arithmetic never yields a signalling NaN, so an FP64 atomic sum
// cannot carry it).
constexpr unsigned long long kOwnMark = 0x7FF00000514D0001ull;

__device__ __forceinline__ void store_own_sum(double2 *slot, float2 S) {
    reinterpret_cast<float2 *>(slot)[0] = S;
    reinterpret_cast<unsigned long long *>(slot)[1] = kOwnMark;
}

// The C64 group sum of a slot: the FP32 sum of its run's thread, else the
// FP64 atomic sum rounded once.
__device__ __forceinline__ float2 group_sum_f2(double2 d) {
    if ((unsigned long long)__double_as_longlong(d.y) == kOwnMark) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(d.x);
        return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
    }
    return to_f2(d);
}

// Dynamic shared memory of the stream kernel for a tile of S stored paths
// (16-byte aligned arrays).  A tile holds at most NG = S + NX - 1 groups: every
// group has a member in the tile, except sub-groups of the tile's last run
// whose members all lie past the tile end (at most NX - 1 of them).
//   gS    [NG] group sums (16 B each)   grep [NG] representative keys
//   wm    [NG] maximum weight (bits)    key/amp [S] the tile's stored paths
//   stage [NSTG][M*M] children amplitudes of the first NSTG groups (S/2
//         for M = 2, S/3 otherwise) between the two passes (tiles usually
//         hold fewer groups; later ones are recomputed in pass B)
//   seg   [S+1] run heads               xm/sb [S]/[S+1] sub-group bits and
//   keep  [NG] survivor bits                 slot bases per run (NX > 1)
//   slot  [NG] run << 4 | x of each sub-group slot (NX > 1)
//   xmask [S][NX] members of each sub-group by offset in its run (offsets
//         below 32; NX > 1), in the staging buffer, which is free until pass A
// key/amp hold S + 32 entries: the 32 paths past the tile end follow the tile.
// followed at run time by the history tables when they are staged.
template <int M, bool C64, int NX, int S>
struct StreamLayout {
    using AmpT = typename std::conditional<C64, float2, double2>::type;
    using WT = typename std::conditional<C64, unsigned, unsigned long long>::type;
    static constexpr int MM = M * M;
    static constexpr int NG = S + NX - 1;
    static constexpr size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    static constexpr int NSTG = M == 2 ? S / 2 : S / 3;
    static constexpr bool stage = (size_t)NSTG * MM * sizeof(AmpT) <= 64 * 1024;
    static constexpr size_t gS = 0;
    static constexpr size_t grep = gS + a16((size_t)NG * sizeof(double2));
    static constexpr size_t wm = grep + a16((size_t)NG * 8);
    static constexpr size_t key = wm + a16((size_t)NG * sizeof(WT));
    static constexpr size_t amp = key + a16((size_t)(S + 32) * 8);
    static constexpr size_t stg = amp + a16((size_t)(S + 32) * sizeof(AmpT));
    static constexpr size_t seg = stg + (stage ? a16((size_t)NSTG * MM * sizeof(AmpT)) : 0);
    static constexpr size_t xm = seg + a16((size_t)(S + 1) * 4);
    static constexpr size_t sb = xm + (NX > 1 ? a16((size_t)S * 4) : 0);
    static constexpr size_t keep = sb + (NX > 1 ? a16((size_t)(S + 1) * 4) : 0);
    static constexpr size_t slot = keep + a16((size_t)NG * 2);
    static constexpr size_t lut = slot + (NX > 1 ? a16((size_t)NG * 4) : 0);
    static constexpr size_t bytes = lut;   // + staged history tables (run time)
};

// Batches of the stream engine: the step's tile size (the smallest multiple
// of NT, up to EPT NT, whose tiles do not outnumber the blocks) into *s_St
// and the first tile of each of the R regions into s_t0[0 .. R] (exclusive
// scan of the regions' tile counts, R <= 2048); block 0 also empties the
// output regions of instances without tiles (otherwise an instance's last
// tile writes its sizes).  All threads; ends with a barrier.
template <int NT, int EPT>
__device__ __forceinline__ void stream_batch_tiles(const unsigned long long *rn_in, unsigned long long *rn_out, int R,
                                                   int MM, int *s_t0, int *s_St) {
    constexpr int NW = NT / 32;
    constexpr int RPT = 2048 / NT;   // regions per thread at most
    __shared__ unsigned long long s_ks[EPT];
    __shared__ unsigned s_ws[NW];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int rpt = (R + NT - 1) / NT;
    const int r0 = (int)threadIdx.x * rpt;
    unsigned q[RPT];   // tiles of NT paths per region
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int r = r0 + u;
        q[u] = (u < rpt && r < R) ? (unsigned)((__ldcg(rn_in + r) + NT - 1) / NT) : 0u;
    }
    if ((int)threadIdx.x < EPT) s_ks[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 1; k < EPT; ++k) {   // tiles at k NT paths per tile
        unsigned long long tk = 0;
#pragma unroll
        for (int u = 0; u < RPT; ++u) tk += (q[u] + k - 1) / k;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tk += __shfl_down_sync(0xffffffffu, tk, o);
        if (lane == 0 && tk) atomicAdd(&s_ks[k], tk);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int St = EPT * NT;
        for (int k = 1; k < EPT; ++k)
            if (s_ks[k] <= (unsigned long long)gridDim.x) {
                St = k * NT;
                break;
            }
        *s_St = St;
    }
    __syncthreads();
    const unsigned kst = (unsigned)(*s_St / NT);
    unsigned cnt[RPT], lsum = 0;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        cnt[u] = (q[u] + kst - 1) / kst;
        lsum += cnt[u];
    }
    unsigned inc = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += y;
    }
    if (lane == 31) s_ws[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0;
        for (int w = 0; w < NW; ++w) {
            const unsigned v = s_ws[w];
            s_ws[w] = a;
            a += v;
        }
        s_t0[R] = (int)a;
    }
    __syncthreads();
    unsigned pos = s_ws[warp] + inc - lsum;
#pragma unroll
    for (int u = 0; u < RPT; ++u)
        if (u < rpt && r0 + u < R) {
            s_t0[r0 + u] = (int)pos;
            pos += cnt[u];
        }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < R / MM; i += NT)
            if (s_t0[i * MM] == s_t0[(i + 1) * MM])
                for (int c = 0; c < MM; ++c) rn_out[i * MM + c] = 0;
}

// Relaxed GPU-scope load of a word other blocks publish (no L1, no
// hoisting; independent loads stay in flight together).
__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// One step of the stream engine: one kernel over tiles of the stored set.
// The set lives in M*M regions (newest point), each sorted by the older
// points, so the paths of one pre-merge group form a run of equal prefix
// (positions 0 .. k-1 of P'); at most one extra position of P' splits a run
// into NX sub-groups.  Per tile (dynamic tickets): load (and prefetch the 32
// paths past the tile end), find run heads; for NX > 1 give each sub-group
// present a compact slot; sum each group and elect its representative, one
// owner thread per group (runs start in the tile and may extend past it;
// runs longer than 32 paths use shared FP64 atomics); compute
// the children of every group once, keep them in shared memory, count the
// survivors per new point and accumulate rho(t+1); get the tile's output
// offsets per region by a decoupled look-back (one warp, a window of
// 32 * LB_K predecessors per round, bounded waits); write the survivors.
// Output region c receives, in order, the children with newest point c of
// all groups, so the next set is again sorted.  No atomics on the data.  The
// last block to finish sums the blocks' partials of rho(t+1) and publishes
// the step.  lut_smem: the history tables of this window length are copied
// into shared memory once per block.
template <int M, bool C64, int NX, int S, bool BATCH>
__device__ __forceinline__ void stream_step_body(const Params &P, int lut_smem) {
    using X = Expander<M, C64>;
    using Lay = StreamLayout<M, C64, NX, S>;
    using AmpT = typename X::AmpT;
    using WT = typename Lay::WT;   // weight |a|^2 as ordered bits: FP32 (C64) or FP64
    constexpr int MM = M * M;
    constexpr int NT = kStreamThreads, NW = NT / 32, EPT = S / NT;
    constexpr int NG = Lay::NG;
    static_assert(S % NT == 0 && EPT <= 32, "tile size");
    static_assert(NX <= 16, "slot map: 4 bits of x");
    static_assert(NW == kStreamWarps, "warp partials");
    static_assert(!BATCH || NX == 1, "batches: P' a prefix of the window");
    constexpr bool kTileAccS = !BATCH && M * M >= 9 && C64;   // per-warp tile sums of rho (see the accumulators)
    DevState *st = P.st;
    // (device state read through L2: the persistent batch kernel runs
    // several steps in one launch)
    if (__ldcg(&st->err)) return;
    const unsigned long long t = __ldcg(&st->t), tn = t + 1;
    if (__ldcg(&st->reg_done) == tn) return;   // the regular kernel just took this step (its new t + 1)
    if constexpr (BATCH) finish_pending_rho_batch(P, st, M * M, false);   // blocks b < n_inst: instance b
    else if (blockIdx.x == 0) finish_pending_rho<C64>(P, st, M * M);   // rho of the previous step
    const int in = (int)(t & 1), outp = (int)(tn & 1), cs = (int)(tn % 3);
    const bool merge = tn >= (unsigned long long)P.dkmax;
    const unsigned long long pref = merge ? P.prefmask : ~0ull;   // filling: every path is its own group
    const int n_act = (int)min(tn, (unsigned long long)P.dkmax);
    const int L_child = (int)min(tn + 1, (unsigned long long)P.dkmax);
    const unsigned long long wmask = (P.b * L_child >= 64) ? ~0ull : ((1ull << (P.b * L_child)) - 1ull);
    const long long G = P.region_cap;
    const unsigned epoch = (unsigned)tn;
    const unsigned long long *keys_in = P.keys[in];
    const AmpT *amps_in = static_cast<const AmpT *>(P.amps[in]);
    unsigned long long *keys_out = P.keys[outp];
    AmpT *amps_out = static_cast<AmpT *>(P.amps[outp]);

    extern __shared__ __align__(16) unsigned char s_dyn[];
    double2 *s_gS = reinterpret_cast<double2 *>(s_dyn + Lay::gS);
    unsigned long long *s_grep = reinterpret_cast<unsigned long long *>(s_dyn + Lay::grep);
    WT *s_wm = reinterpret_cast<WT *>(s_dyn + Lay::wm);
    unsigned long long *s_key = reinterpret_cast<unsigned long long *>(s_dyn + Lay::key);
    AmpT *s_amp = reinterpret_cast<AmpT *>(s_dyn + Lay::amp);
    AmpT *s_stg = reinterpret_cast<AmpT *>(s_dyn + Lay::stg);
    int *s_seg = reinterpret_cast<int *>(s_dyn + Lay::seg);
    unsigned *s_xm = reinterpret_cast<unsigned *>(s_dyn + Lay::xm);
    int *s_sb = reinterpret_cast<int *>(s_dyn + Lay::sb);
    unsigned short *s_keep = reinterpret_cast<unsigned short *>(s_dyn + Lay::keep);
    int *s_slot = reinterpret_cast<int *>(s_dyn + Lay::slot);
    unsigned *s_xmask = reinterpret_cast<unsigned *>(s_dyn + Lay::stg);
    static_assert(NX == 1 || (Lay::stage && (size_t)Lay::NSTG * MM * sizeof(AmpT) >= (size_t)S * NX * 4),
                  "sub-group member masks live in the staging buffer");
    __shared__ double2 s_w[C64 || BATCH ? 1 : MM * MM];   // FP64 weights (FP64 path only)
    __shared__ float4 s_wf[BATCH ? 1 : MM * MM];
    __shared__ long long s_nr[MM], s_tile0[MM + 1];
    __shared__ unsigned s_wsum[NW][MM];
    __shared__ unsigned long long s_base[MM], s_tot[MM], s_kprev;
    __shared__ unsigned s_ra_n;   // prefetched paths past the tile end
    __shared__ long long s_ahead;   // tile-relative end of the tile's last run
    __shared__ unsigned s_ticket, s_nseg, s_ng, s_hw[NW];
    __shared__ int s_St;   // tile size of this step
    __shared__ float4 s_rt[NW][MM];
    __shared__ float4 s_wrho[kTileAccS ? NW : 1][MM];   // M >= 3 single problems: per-warp sums of rho(t+1)
    __shared__ bool s_last;
    __shared__ int s_any;   // the block processed a tile
    __shared__ int s_lbfail;   // the tile's look-back gave up (timeout, or another block's error)
    const double tie_d = 1.0 - P.tie_rel;   // R4 window, once per thread
    const unsigned stall = __ldcg(&st->stall_tile);   // test hook (0 in normal operation)
    // batches: R = n_inst * M*M regions (instance, newest point); behind the
    // tile buffers (no staged tables) each instance's block sums of rho and
    // survivors, [n_inst][M*M + 1], and the first tile of every region
    const int R = BATCH ? P.n_inst * MM : MM;
    double2 *s_acc = reinterpret_cast<double2 *>(s_dyn + Lay::lut);
    int *s_t0 = reinterpret_cast<int *>(s_dyn + Lay::lut + (((size_t)(BATCH ? P.n_inst : 1) * (MM + 1) * 16 + 15) & ~(size_t)15));
    const float tie_f = (float)tie_d;

    // weights and the history tables of this window length (batches read
    // their instance's from global memory per tile)
    if constexpr (!BATCH)
        for (int i = threadIdx.x; i < MM * MM; i += NT) {
            if constexpr (!C64) s_w[i] = P.wtab[i];
            s_wf[i] = P.wtabf[i];
        }
    Tab tab = tab_global(P, n_act, 0);
    // (asynchronous copies, waited for before the first pass A: the tables
    // arrive while the first tile loads; rows are whole multiples of
    // kLutEntries entries, so every copy is 16-byte aligned)
    if (!BATCH && lut_smem && P.ndelta) {
        const int n = P.nchunks * kLutEntries;
        if constexpr (C64) {
            float2 *hi = reinterpret_cast<float2 *>(s_dyn + Lay::lut), *lo = hi + n;
            for (int i = threadIdx.x; i < n / 2; i += NT) {
                cp_async16(hi + 2 * i, tab.hi + 2 * i);
                cp_async16(lo + 2 * i, tab.lo + 2 * i);
            }
            tab.hi = hi;
            tab.lo = lo;
        } else {
            double2 *et = reinterpret_cast<double2 *>(s_dyn + Lay::lut);
            for (int i = threadIdx.x; i < n * P.ndelta; i += NT) cp_async16(et + i, tab.et + i);
            tab.et = et;
        }
    }
    if (threadIdx.x == 0) s_any = 0;
    if constexpr (kTileAccS)
        for (int i = threadIdx.x; i < NW * MM; i += NT) (&s_wrho[0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (BATCH) {
        for (int i = threadIdx.x; i < P.n_inst * (MM + 1); i += NT) s_acc[i] = make_double2(0.0, 0.0);
        stream_batch_tiles<NT, EPT>(P.reg_n + (size_t)in * R, P.reg_n + (size_t)outp * R, R, MM, s_t0, &s_St);
    } else if (threadIdx.x == 0) {
        for (int r = 0; r < MM; ++r) s_nr[r] = (long long)__ldcg(&P.reg_n[in * MM + r]);
        // tile size of this step: the smallest multiple of NT (up to S) whose
        // tiles do not outnumber the blocks, so that a small step runs in one
        // wave of short tiles (a large one uses S)
        // (ceil(n / (k NT)) = ceil(ceil(n / NT) / k): 32-bit divisions by k)
        unsigned q[MM];
        for (int r = 0; r < MM; ++r) q[r] = (unsigned)((s_nr[r] + NT - 1) / NT);
        int St = S;
        for (unsigned k = 1; k < (unsigned)EPT; ++k) {
            long long tiles = 0;
            for (int r = 0; r < MM; ++r) tiles += (q[r] + k - 1) / k;
            if (tiles <= (long long)gridDim.x) {
                St = (int)k * NT;
                break;
            }
        }
        s_St = St;
        const unsigned kst = (unsigned)(St / NT);
        long long acc = 0;
        for (int r = 0; r < MM; ++r) {
            s_tile0[r] = acc;
            acc += (q[r] + kst - 1) / kst;
        }
        s_tile0[MM] = acc;
        if (acc == 0 && blockIdx.x == 0) {   // empty input: the output is empty
            for (int r = 0; r < MM; ++r) P.reg_n[outp * MM + r] = 0;
            st->cnt_out[cs] = 0;
        }
    }
    __syncthreads();
    const long long ntiles = BATCH ? (long long)s_t0[R] : s_tile0[MM];
    // region of a tile (the last region whose first tile is at or before it),
    // its first tile and its stored paths
    auto region_of = [&](long long tk) -> int {
        if constexpr (BATCH) {
            int lo = 0, hi = R;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if ((long long)s_t0[mid] <= tk) lo = mid;
                else hi = mid;
            }
            return lo;
        } else {
            int rr = 0;
            while (rr + 1 < MM && tk >= s_tile0[rr + 1]) ++rr;
            return rr;
        }
    };
    auto tile0_of = [&](int rr) -> long long {
        if constexpr (BATCH) return (long long)s_t0[rr];
        else return s_tile0[rr];
    };
    auto nr_of = [&](int rr) -> long long {
        if constexpr (BATCH) return (long long)__ldcg(P.reg_n + (size_t)in * R + rr);
        else return s_nr[rr];
    };
    const int St = s_St, ept = St / NT;   // entries per thread this step (<= EPT)
    // rho(t+1) accumulators of this thread: FP64, or on the C64 path FP32
    // with a Kahan compensation term (M = 2; plain FP32 sums for M >= 3).
    // Single problems keep them for the whole kernel and widen them once at
    // the end, except C64 with M >= 3 (two blocks per SM, 128 registers:
    // kept across the tile loop, the M*M accumulators were spilled and every
    // child's addition went through local memory), where they live for one
    // tile's write pass and a warp sum per tile is added to a per-warp FP32
    // pair (TwoSum).  Batches sum them per tile into their instance's block
    // sums
    constexpr bool kKahan = C64 && M == 2;
    constexpr bool kTileAcc = BATCH || kTileAccS;
    typename X::AccT racc[kTileAcc ? 1 : MM], rcmp[kKahan && !kTileAcc ? MM : 1];
    if constexpr (!kTileAcc) {
#pragma unroll
        for (int k = 0; k < MM; ++k) {
            racc[k].x = racc[k].y = 0;
            if constexpr (kKahan) rcmp[k].x = rcmp[k].y = 0;
        }
    }
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned long long block_kept = 0;
    auto weight_bits = [&](AmpT a) -> WT {
        if constexpr (C64) return __float_as_uint(a.x * a.x + a.y * a.y);
        else return (unsigned long long)__double_as_longlong(a.x * a.x + a.y * a.y);
    };
    auto within_tie = [&](WT w, WT wm) -> bool {
        if constexpr (C64) return __uint_as_float(w) >= tie_f * __uint_as_float(wm);
        else return __longlong_as_double((long long)w) >= tie_d * __longlong_as_double((long long)wm);
    };
    auto xval = [&](unsigned long long key) -> unsigned {
        return NX > 1 ? (unsigned)((key >> P.x_shift) & (NX - 1)) : 0u;
    };
    // first wave: block b prefetches tile b's stored paths into L2 (one
    // address inside the tile per 128-byte line of keys and amplitudes), so
    // that whichever block takes tile b finds it there
    if ((long long)blockIdx.x < ntiles) {
        const long long tk = blockIdx.x;
        const int rr = region_of(tk);
        const long long b0 = (tk - tile0_of(rr)) * St;
        const long long n = min((long long)St, nr_of(rr) - b0);
        const char *kp = reinterpret_cast<const char *>(keys_in + rr * G + b0);
        const char *ap = reinterpret_cast<const char *>(amps_in + rr * G + b0);
        const int kl = (int)((n * 8 + 127) / 128), al = (int)((n * (long long)sizeof(AmpT) + 127) / 128);
        for (int l = threadIdx.x; l < kl + al; l += NT) {
            const char *a = l < kl ? kp + (size_t)l * 128 : ap + (size_t)(l - kl) * 128;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
        }
    }

    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&st->ticket[cs], 1u);
        __syncthreads();
        const long long ticket = s_ticket;
        if (ticket >= ntiles) break;
        if (threadIdx.x == 0) s_any = 1;
        const int r = region_of(ticket);
        const long long e0 = (ticket - tile0_of(r)) * St;
        const long long nr = nr_of(r);
        // the tile's instance (batches): its tables, its first output region
        // and the tiles of its regions, which bound the look-back
        const int inst = BATCH ? r / MM : 0, rb = BATCH ? inst * MM : 0;
        Tab tab_t = tab;
        const double2 *w_t = s_w;
        const float4 *wf_t = s_wf;
        long long lb0 = 0, tlast = ntiles - 1;
        if constexpr (BATCH) {
            tab_t = tab_global(P, n_act, inst);
            w_t = P.wtab + (size_t)inst * MM * MM;
            wf_t = P.wtabf + (size_t)inst * MM * MM;
            lb0 = s_t0[rb];
            tlast = (long long)s_t0[rb + MM] - 1;
        }
        const int cnt = (int)min((long long)St, nr - e0);
        const unsigned long long *kin = keys_in + r * G;
        const AmpT *ain = amps_in + r * G;
        // load the tile; warp 0 prefetches the 32 paths past its end (the
        // last run may continue there), thread 0 the key before it; slots of
        // the previous tile are free (the loop ends with a barrier)
        // (16-byte asynchronous copies, all in flight at once, no registers:
        // region bases and tile starts are 16-entry aligned; a ragged end
        // reads only its entries; waited for before the barrier below)
        {
            const int kc = (cnt * 8 + 15) / 16, ac = (cnt * (int)sizeof(AmpT) + 15) / 16;
            const char *kg = reinterpret_cast<const char *>(kin + e0), *ag = reinterpret_cast<const char *>(ain + e0);
            char *ks = reinterpret_cast<char *>(s_key), *as = reinterpret_cast<char *>(s_amp);
            for (int c = threadIdx.x; c < kc + ac; c += NT) {
                if (c < kc) cp_async16_part(ks + 16 * c, kg + 16 * c, (unsigned)min(16, cnt * 8 - 16 * c));
                else {
                    const int d = c - kc;
                    cp_async16_part(as + 16 * d, ag + 16 * d, (unsigned)min(16, cnt * (int)sizeof(AmpT) - 16 * d));
                }
            }
        }
        if (warp == 0) {
            const bool ok = cnt == St && e0 + St + lane < nr;
            if (ok) {
                s_key[St + lane] = __ldcg(kin + e0 + St + lane);
                s_amp[St + lane] = __ldcg(ain + e0 + St + lane);
            }
            const unsigned okm = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) s_ra_n = __popc(okm);   // a prefix of the 32 lanes
        }
        if (threadIdx.x == 0) s_kprev = e0 > 0 ? __ldcg(kin + e0 - 1) : 0ull;
        for (int i = threadIdx.x; i < NG; i += NT) {
            s_gS[i] = make_double2(0.0, 0.0);
            s_grep[i] = kEmpty;
            s_wm[i] = 0;
        }
        if constexpr (NX > 1) {
            for (int i = threadIdx.x; i < S; i += NT) s_xm[i] = 0u;
            for (int i = threadIdx.x; i < St * NX / 4; i += NT) reinterpret_cast<uint4 *>(s_xmask)[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        cp_async_wait_all();   // the tile's copies (and, at the first tile, the staged tables)
        __syncthreads();
        // run heads (ept consecutive entries per thread), block scan of their count
        unsigned hmask = 0;
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
            const int i = threadIdx.x * ept + u;
            if (u < ept && i < cnt) {
                if (i == 0 && e0 == 0) hmask |= 1u << u;
                else if ((s_key[i] & pref) != ((i > 0 ? s_key[i - 1] : s_kprev) & pref)) hmask |= 1u << u;
            }
        }
        const unsigned hc = __popc(hmask);
        unsigned hincl = hc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, hincl, o);
            if ((int)lane >= o) hincl += y;
        }
        if (lane == 31) s_hw[warp] = hincl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned a = 0;
            for (int w = 0; w < NW; ++w) {
                const unsigned v = s_hw[w];
                s_hw[w] = a;
                a += v;
            }
            s_nseg = a;
        }
        __syncthreads();
        const int nseg = (int)s_nseg;
        const int segbase = (int)(s_hw[warp] + hincl - hc) - 1;   // run of the entry before the thread's first
        {
            int pos = segbase + 1;
#pragma unroll
            for (int u = 0; u < EPT; ++u)
                if (hmask & (1u << u)) s_seg[pos++] = threadIdx.x * ept + u;
        }
        __syncthreads();
        // extent of the tile's last run past the tile end (warp 0): members
        // share its prefix; the first 32 come from the prefetch.  For NX > 1
        // the sub-group bits of every run are collected.
        const unsigned long long plast = nseg ? (s_key[s_seg[nseg - 1]] & pref) : 0ull;
        long long ahead = cnt;   // tile-relative end of the last run
        if constexpr (NX > 1) {
            int sg = segbase, rs = segbase >= 0 ? s_seg[segbase] : 0;   // run and its start
#pragma unroll
            for (int u = 0; u < EPT; ++u) {
                const int i = threadIdx.x * ept + u;
                if (hmask & (1u << u)) {
                    ++sg;
                    rs = i;
                }
                if (u < ept && i < cnt && sg >= 0) {
                    const unsigned x = xval(s_key[i]);
                    if (i - rs < 32) atomicOr(&s_xmask[sg * NX + x], 1u << (i - rs));
                    else atomicOr(&s_xm[sg], 1u << x);
                }
            }
        }
        if (warp == 0 && nseg > 0 && cnt == St) {
            unsigned long long key = s_key[cnt + lane];
            bool inrun = lane < s_ra_n && (key & pref) == plast;
            for (int round = 0;; ++round) {
                if (round > 0) {
                    const long long i = e0 + ahead + lane;
                    inrun = i < nr;
                    if (inrun) {
                        key = __ldcg(kin + i);
                        inrun = (key & pref) == plast;
                    }
                }
                const unsigned inm = __ballot_sync(0xffffffffu, inrun);
                const int nin = inm == 0xffffffffu ? 32 : __ffs(~inm) - 1;   // leading members of the run
                if constexpr (NX > 1) {
                    if ((int)lane < nin) {
                        const long long off = ahead + lane - s_seg[nseg - 1];
                        if (off < 32) atomicOr(&s_xmask[(nseg - 1) * NX + xval(key)], 1u << off);
                        else atomicOr(&s_xm[nseg - 1], 1u << xval(key));
                    }
                }
                ahead += nin;
                if (nin < 32) break;
            }
        }
        if (threadIdx.x == 0) s_ahead = ahead;
        __syncthreads();
        ahead = s_ahead;
        // compact slots: sub-groups of run sg are slots sb[sg] + rank of x
        int ngroups = nseg;
        if constexpr (NX > 1) {
            // rpt consecutive runs per thread: thread-local sum, warp scan,
            // across warps.  A run's sub-groups: its members at offsets
            // below 32 (masks) and beyond (xm bits); the union goes back to xm.
            const int rpt = (nseg + NT - 1) / NT;
            unsigned xmv[EPT];
            unsigned lsum = 0;
#pragma unroll
            for (int u = 0; u < EPT; ++u) {
                const int g = threadIdx.x * rpt + u;
                xmv[u] = 0u;
                if (u < rpt && g < nseg) {
                    xmv[u] = s_xm[g];
#pragma unroll
                    for (int x = 0; x < NX; ++x) xmv[u] |= (s_xmask[g * NX + x] != 0u ? 1u : 0u) << x;
                }
                lsum += (unsigned)__popc(xmv[u]);
            }
            unsigned inc = lsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if ((int)lane >= o) inc += y;
            }
            if (lane == 31) s_wsum[warp][0] = inc;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned a = 0;
                for (int w = 0; w < NW; ++w) {
                    const unsigned v = s_wsum[w][0];
                    s_wsum[w][0] = a;
                    a += v;
                }
                s_ng = a;
            }
            __syncthreads();
            unsigned pos = s_wsum[warp][0] + inc - lsum;
#pragma unroll
            for (int u = 0; u < EPT; ++u) {
                const int g = threadIdx.x * rpt + u;
                if (u < rpt && g < nseg) {
                    s_sb[g] = (int)pos;
                    s_xm[g] = xmv[u];
                }
                for (unsigned m = xmv[u]; m; m &= m - 1u) s_slot[pos++] = (g << 4) | (__ffs(m) - 1);
            }
            ngroups = (int)s_ng;
            __syncthreads();
        }
        auto slot_of = [&](int sg, unsigned long long key) -> int {
            if constexpr (NX > 1) {
                const unsigned m = s_xm[sg];
                return s_sb[sg] + __popc(m & ((1u << xval(key)) - 1u));
            } else {
                return sg;
            }
        };
        // groups of runs of at most kOwnRun members (all runs once the window
        // is full) have one owner thread each, which visits the group's
        // members (the whole run, or for NX > 1 the sub-group's mask) twice
        // in order: walk 1 adds them (C64: FP32 with the rounding error of
        // every addition kept, TwoSum, rounded once; FP64: FP64) and takes
        // their maximum weight, walk 2 elects the representative.  No atomics
        // and no stores in the loops; the result does not depend on the
        // tiling.  FP64 sub-groups (NX > 1) stay with the shared atomics
        // below, one entry per thread, which keeps the FP64 pipe (1/64 of the
        // FP32 rate) to one addition per member.
        constexpr bool kOwners = NX == 1 || C64;
        bool any_long = !kOwners && nseg > 0;
        cp_async_wait_all();   // staged history tables (first tile), published by the barrier below
        if constexpr (kOwners) {
            const int nown = NX > 1 ? ngroups : nseg;
            for (int sl = threadIdx.x; sl < nown; sl += NT) {
                int g = sl;
                unsigned x = 0;
                if constexpr (NX > 1) {
                    const int gx = s_slot[sl];
                    g = gx >> 4;
                    x = (unsigned)gx & 15u;
                }
                const int b0 = s_seg[g];
                const long long b1 = g + 1 < nseg ? (long long)s_seg[g + 1] : ahead;
                if (b1 - b0 > kOwnRun) {
                    any_long = true;
                    continue;
                }
                const int n = (int)b1 - b0;   // members past the tile end are in the prefetch
                typename X::AccT sh, se;
                sh.x = sh.y = 0;
                se.x = se.y = 0;
                WT wmx = 0;
                auto add = [&](const AmpT &a) {
                    if constexpr (C64) {
                        two_sum_acc(sh.x, se.x, a.x);
                        two_sum_acc(sh.y, se.y, a.y);
                    } else {
                        sh.x += a.x;
                        sh.y += a.y;
                    }
                    const WT wb = weight_bits(a);
                    wmx = wb > wmx ? wb : wmx;
                };
                unsigned mm;   // the group's members by offset in the run
                if constexpr (NX > 1) {
                    mm = s_xmask[g * NX + x];
#pragma unroll 4
                    for (unsigned m = mm; m; m &= m - 1u) add(s_amp[b0 + __ffs(m) - 1]);
                } else {
                    mm = n == 32 ? 0xffffffffu : (1u << n) - 1u;
#pragma unroll 4
                    for (int j = 0; j < n; ++j) add(s_amp[b0 + j]);
                }
                unsigned long long kmin = kEmpty;
                for (unsigned m = mm; m; m &= m - 1u) {
                    const int i = b0 + __ffs(m) - 1;
                    const unsigned long long key = s_key[i];
                    if (within_tie(weight_bits(s_amp[i]), wmx) && key < kmin) kmin = key;
                }
                if constexpr (C64) store_own_sum(s_gS + sl, make_float2(sh.x + se.x, sh.y + se.y));
                else s_gS[sl] = make_double2(sh.x, sh.y);
                s_grep[sl] = kmin;
            }
        }
        // longer runs (only while the window fills): every member adds to its
        // group in FP64 with shared atomics (consecutive members of a thread
        // in the same slot combined first), then, after a barrier, the members
        // within the tie window compete for the representative
        if (__syncthreads_or(any_long)) {
            auto run_long = [&](int g) -> bool {
                if constexpr (!kOwners) return true;
                const long long b1 = g + 1 < nseg ? (long long)s_seg[g + 1] : ahead;
                return b1 - s_seg[g] > kOwnRun;
            };
            const bool last_long = nseg > 0 && run_long(nseg - 1);
            {
                int sg = segbase, cur = -1;
                bool lng = sg >= 0 && run_long(sg);
                double ax = 0.0, ay = 0.0;
                WT wmx = 0;
#pragma unroll
                for (int u = 0; u < EPT; ++u) {
                    const int i = threadIdx.x * ept + u;
                    if (hmask & (1u << u)) lng = run_long(++sg);
                    if (u < ept && i < cnt && lng) {
                        const AmpT a = s_amp[i];
                        const int sl = slot_of(sg, s_key[i]);
                        const WT wb = weight_bits(a);
                        if (sl != cur) {
                            if (cur >= 0) {
                                atomicAdd(&s_gS[cur].x, ax);
                                atomicAdd(&s_gS[cur].y, ay);
                                atomicMax(&s_wm[cur], wmx);
                            }
                            cur = sl;   // the slot's local sum starts at its first member
                            ax = to_d(a.x);
                            ay = to_d(a.y);
                            wmx = wb;
                        } else {
                            ax += to_d(a.x);
                            ay += to_d(a.y);
                            wmx = wb > wmx ? wb : wmx;
                        }
                    }
                }
                if (cur >= 0) {
                    atomicAdd(&s_gS[cur].x, ax);
                    atomicAdd(&s_gS[cur].y, ay);
                    atomicMax(&s_wm[cur], wmx);
                }
            }
            if (warp == 0 && last_long && ahead > cnt) {   // members of the last run past the tile end
                for (long long base = cnt; base < ahead; base += 32) {
                    const long long i = base + lane;
                    if (i < ahead) {
                        unsigned long long key;
                        AmpT a;
                        if (base == cnt) {
                            key = s_key[cnt + lane];
                            a = s_amp[cnt + lane];
                        } else {
                            key = __ldcg(kin + e0 + i);
                            a = __ldcg(ain + e0 + i);
                        }
                        const int sl = slot_of(nseg - 1, key);
                        atomicAdd(&s_gS[sl].x, to_d(a.x));
                        atomicAdd(&s_gS[sl].y, to_d(a.y));
                        atomicMax(&s_wm[sl], weight_bits(a));
                    }
                }
            }
            __syncthreads();
            {
                int sg = segbase, cur = -1;
                bool lng = sg >= 0 && run_long(sg);
                unsigned long long kmin = kEmpty;
#pragma unroll
                for (int u = 0; u < EPT; ++u) {
                    const int i = threadIdx.x * ept + u;
                    if (hmask & (1u << u)) lng = run_long(++sg);
                    if (u < ept && i < cnt && lng) {
                        const unsigned long long key = s_key[i];
                        const int sl = slot_of(sg, key);
                        if (sl != cur) {
                            if (cur >= 0 && kmin != kEmpty) atomicMin(&s_grep[cur], kmin);
                            cur = sl;
                            kmin = kEmpty;
                        }
                        if (within_tie(weight_bits(s_amp[i]), s_wm[sl]) && key < kmin) kmin = key;
                    }
                }
                if (cur >= 0 && kmin != kEmpty) atomicMin(&s_grep[cur], kmin);
            }
            if (warp == 0 && last_long && ahead > cnt) {
                for (long long base = cnt; base < ahead; base += 32) {
                    const long long i = base + lane;
                    if (i < ahead) {
                        unsigned long long key;
                        AmpT a;
                        if (base == cnt) {
                            key = s_key[cnt + lane];
                            a = s_amp[cnt + lane];
                        } else {
                            key = __ldcg(kin + e0 + i);
                            a = __ldcg(ain + e0 + i);
                        }
                        const int sl = slot_of(nseg - 1, key);
                        if (within_tie(weight_bits(a), s_wm[sl])) atomicMin(&s_grep[sl], key);
                    }
                }
            }
            __syncthreads();
        }
        // pass A: children of a contiguous range of groups per thread, once;
        // survivors counted per new point, amplitudes kept in shared memory
        // for pass B (the first NSTG groups)
        // (contiguous ranges in thread order, so that the survivors are written
        // in group order; the first ngroups % NT threads take one more)
        const int gq = ngroups / NT, gr = ngroups - gq * NT;
        const int g0 = (int)threadIdx.x * gq + min((int)threadIdx.x, gr);
        const int g1 = g0 + gq + ((int)threadIdx.x < gr ? 1 : 0);
        unsigned cntc[MM];
#pragma unroll
        for (int c = 0; c < MM; ++c) cntc[c] = 0;
        for (int g = g0; g < g1; ++g) {
            const unsigned long long rk = s_grep[g];
            unsigned keep = 0;
            AmpT v[MM];
            if (rk != kEmpty) {
                if constexpr (C64) {
                    const float2 Sf = group_sum_f2(s_gS[g]);
                    reinterpret_cast<float2 *>(s_gS)[2 * g] = Sf;   // for pass B, if not staged
                    keep = X::children_tab(P, tab_t, rk, Sf, w_t, wf_t, v);
                } else {
                    keep = X::children_tab(P, tab_t, rk, s_gS[g], w_t, wf_t, v);
                }
            }
            s_keep[g] = (unsigned short)keep;
#pragma unroll
            for (int c = 0; c < MM; ++c) {
                if (!(keep & (1u << c))) continue;
                ++cntc[c];
                if (Lay::stage && g < Lay::NSTG) s_stg[g * MM + c] = v[c];
            }
        }
        // block exclusive scan per new point (warp shuffles, then across warps)
        unsigned tb[MM];
#pragma unroll
        for (int c = 0; c < MM; ++c) {
            unsigned v = cntc[c], incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            tb[c] = incl - v;
            if (lane == 31) s_wsum[warp][c] = incl;
        }
        __syncthreads();
        if (threadIdx.x < MM) {
            unsigned a = 0;
            for (int w = 0; w < NW; ++w) {
                const unsigned v = s_wsum[w][threadIdx.x];
                s_wsum[w][threadIdx.x] = a;
                a += v;
            }
            s_tot[threadIdx.x] = a;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < MM; ++c) tb[c] += s_wsum[warp][c];
        // M >= 3: the thread's offsets wait in the tile's key and amplitude
        // buffers (free since pass A, contiguous) while the look-back runs,
        // [c][thread], where they fit
        constexpr bool kTbShared = MM >= 9 && (size_t)MM * NT * 4 <= Lay::stg - Lay::key;
        unsigned *s_tb = reinterpret_cast<unsigned *>(s_dyn + Lay::key);
        if constexpr (kTbShared) {
#pragma unroll
            for (int c = 0; c < MM; ++c) s_tb[c * NT + threadIdx.x] = tb[c];
        }
        // decoupled look-back, one warp per bucket (buckets c, c + NW, ...):
        // publish the tile's aggregate, then read a window of 32 * LBK
        // predecessors: position p = j * 32 + lane is tile pred - p, so each
        // load instruction reads 32 consecutive words of the bucket (relaxed
        // GPU-scope loads).  With u the nearest unpublished and i the nearest
        // inclusive position: i < u ends the look-back (sum up to i);
        // otherwise the published aggregates before u are added and the
        // window moves to u, waiting (bounded) only for that tile.  A wide
        // window matters when all tiles run at once: inclusive prefixes then
        // spread one window per round.
        constexpr int LBK = 4;
        constexpr int WIN = 32 * LBK;
        const bool withhold = stall != 0u && (long long)stall == ticket + 1;   // test hook: publish nothing
        if (threadIdx.x == 0) s_lbfail = 0;
        __syncthreads();
        // buckets c = warp + j * NW (KB per warp: two for M = 3, 4) are
        // looked back in the same rounds: their loads are issued together
        constexpr int KB = (MM + NW - 1) / NW;
        if ((int)warp < MM) {
            unsigned long long excl[KB];
            long long pred[KB];
            bool done[KB];
#pragma unroll
            for (int j = 0; j < KB; ++j) {
                const int c = (int)warp + j * NW;
                excl[j] = 0;
                pred[j] = ticket - 1;
                done[j] = c >= MM || pred[j] < lb0;
                if (c < MM && lane == 0 && !withhold)
                    atomicExch(P.tile_state + (size_t)c * P.max_tiles + ticket,
                               lb_word(epoch, ticket == lb0 ? kLbInc : kLbAgg, s_tot[c]));
            }
            const long long t0 = clock64();
            bool timeout = false, abort = false;   // abort: another block raised an error
            for (;;) {
                unsigned wv[KB][LBK];   // (state << 30) | count of this step; 0: not yet published
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    const unsigned long long *bucket = P.tile_state + (size_t)((int)warp + j * NW) * P.max_tiles;
#pragma unroll
                    for (int k = 0; k < LBK; ++k) {
                        const long long idx = pred[j] - (long long)k * 32 - lane;
                        if (done[j] || idx < lb0) {
                            wv[j][k] = kLbInc << 30;   // before the instance's first tile: an inclusive prefix of 0
                        } else {
                            const unsigned long long w = ld_relaxed_gpu(bucket + idx);
                            wv[j][k] = (unsigned)(w >> 32) == epoch ? (unsigned)w : 0u;
                        }
                    }
                }
                bool wait = false, all = true;
#pragma unroll
                for (int j = 0; j < KB; ++j) {
                    if (done[j]) continue;
                    int u = WIN, i = WIN;   // nearest unpublished / inclusive position
#pragma unroll
                    for (int k = LBK - 1; k >= 0; --k) {
                        const unsigned um = __ballot_sync(0xffffffffu, wv[j][k] == 0u);
                        const unsigned im = __ballot_sync(0xffffffffu, (wv[j][k] >> 30) == kLbInc);
                        if (um) u = k * 32 + __ffs(um) - 1;
                        if (im) i = k * 32 + __ffs(im) - 1;
                    }
                    const bool fin = i < u;
                    const int lim = fin ? i + 1 : u;   // positions summed this round
                    if (lim > 0) {
                        unsigned long long part = 0;
#pragma unroll
                        for (int k = 0; k < LBK; ++k)
                            if (k * 32 + (int)lane < lim) part += wv[j][k] & ((1u << 30) - 1u);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
                        excl[j] += __shfl_sync(0xffffffffu, part, 0);
                    }
                    if (fin) {
                        done[j] = true;
                        continue;
                    }
                    pred[j] -= lim;
                    if (pred[j] < lb0) {
                        done[j] = true;
                        continue;
                    }
                    all = false;
                    if (lim < WIN) wait = true;   // waiting on tile pred[j]: bounded
                }
                if (all) break;
                if (wait) {
                    if (*(volatile unsigned *)&st->err) {
                        abort = true;
                        break;
                    }
                    if (clock64() - t0 > kBarrierCycles) {
                        timeout = true;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            if (timeout && lane == 0) atomicOr(&st->err, kErrTimeout);
            if (lane == 0) {
                if (timeout || abort) {
                    s_lbfail = 1;   // offsets unknown: this tile writes nothing (the step fails)
                } else {
#pragma unroll
                    for (int j = 0; j < KB; ++j) {
                        const int c = (int)warp + j * NW;
                        if (c >= MM) continue;
                        const unsigned long long tot = s_tot[c];
                        if (ticket > lb0 && !withhold)
                            atomicExch(P.tile_state + (size_t)c * P.max_tiles + ticket,
                                       lb_word(epoch, kLbInc, excl[j] + tot));
                        s_base[c] = excl[j];
                        if (ticket == tlast) P.reg_n[(size_t)outp * R + rb + c] = excl[j] + tot;   // the last tile knows the sizes
                    }
                }
            }
        }
        __syncthreads();
        const bool lbfail = s_lbfail != 0;
        if (threadIdx.x == 0 && !lbfail) {
            for (int c = 0; c < MM; ++c) block_kept += s_tot[c];
            if (ngroups) atomicAdd(&st->cnt_groups[cs], (unsigned long long)ngroups);
            if (ticket == tlast) {
                unsigned long long sumc = 0;
                for (int c = 0; c < MM; ++c) sumc += s_base[c] + s_tot[c];
                if constexpr (BATCH) atomicAdd(&st->cnt_out[cs], sumc);   // zeroed by the previous step
                else st->cnt_out[cs] = sumc;
            }
        }
        // pass B: write the survivors to their regions
        if constexpr (kTbShared) {
#pragma unroll
            for (int c = 0; c < MM; ++c) tb[c] = s_tb[c * NT + threadIdx.x];
        }
        typename X::AccT tacc[kTileAcc ? MM : 1], tcmp[kTileAcc && kKahan ? MM : 1];
        if constexpr (kTileAcc) {
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                tacc[k].x = tacc[k].y = 0;
                if constexpr (kKahan) tcmp[k].x = tcmp[k].y = 0;
            }
        }
        for (int g = g0; g < (lbfail ? g0 : g1); ++g) {
            const unsigned keep = s_keep[g];
            if (!keep) continue;
            const unsigned long long rk = s_grep[g];
            AmpT v[MM];
            if (Lay::stage && g < Lay::NSTG) {
#pragma unroll
                for (int c = 0; c < MM; ++c)
                    if (keep & (1u << c)) v[c] = s_stg[g * MM + c];
            } else if constexpr (C64) {
                X::children_tab(P, tab_t, rk, reinterpret_cast<const float2 *>(s_gS)[2 * g], w_t, wf_t, v);
            } else {
                X::children_tab(P, tab_t, rk, s_gS[g], w_t, wf_t, v);
            }
            const unsigned long long shifted = rk << P.b;
#pragma unroll
            for (int c = 0; c < MM; ++c) {
                if (!(keep & (1u << c))) continue;
                const unsigned long long o = s_base[c] + tb[c]++;
                if ((long long)o >= G) {
                    raise_err(st, kErrPaths);
                    continue;
                }
                const unsigned long long code = (unsigned long long)((c / M) | ((c % M) << P.bs));
                keys_out[(rb + c) * G + o] = (shifted | code) & wmask;
                amps_out[(rb + c) * G + o] = v[c];
                if constexpr (kTileAcc) {
                    if constexpr (kKahan) {
                        X::kahan_add(tacc[c], tcmp[c], v[c]);
                    } else {
                        tacc[c].x += v[c].x;
                        tacc[c].y += v[c].y;
                    }
                } else if constexpr (kKahan) {
                    X::kahan_add(racc[c], rcmp[c], v[c]);
                } else {
                    racc[c].x += v[c].x;
                    racc[c].y += v[c].y;
                }
            }
        }
        if constexpr (BATCH) {
            // the tile's part of its instance's rho(t+1) and survivor count:
            // FP64 warp sums added to the block's sums (shared FP64 atomics)
            double2 *acc = s_acc + (size_t)inst * (MM + 1);
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                double x = to_d(tacc[k].x), y = to_d(tacc[k].y);
                if constexpr (kKahan) {
                    x -= to_d(tcmp[k].x);
                    y -= to_d(tcmp[k].y);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_down_sync(0xffffffffu, x, o);
                    y += __shfl_down_sync(0xffffffffu, y, o);
                }
                if (lane == 0 && (x != 0.0 || y != 0.0)) {
                    atomicAdd(&acc[k].x, x);
                    atomicAdd(&acc[k].y, y);
                }
            }
            if (threadIdx.x == 0 && !lbfail) {
                unsigned long long kt = 0;
                for (int c = 0; c < MM; ++c) kt += s_tot[c];
                atomicAdd(&acc[MM].x, (double)kt);
            }
        }
        if constexpr (kTileAccS) {
            // the tile's rho(t+1): warp sums (plain FP32), added by lane 0 to
            // the warp's pair with TwoSum (the error kept)
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                auto x = tacc[k].x, y = tacc[k].y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_down_sync(0xffffffffu, x, o);
                    y += __shfl_down_sync(0xffffffffu, y, o);
                }
                if (lane == 0) {
                    float4 a = s_wrho[warp][k];
                    two_sum_acc(a.x, a.y, x);
                    two_sum_acc(a.z, a.w, y);
                    s_wrho[warp][k] = a;
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();   // a block without a tile: its table copies
    // arrive first: the last block to arrive publishes the step, for which
    // it needs the step's counters only; every block then writes its partial
    // of rho, which the next step's block 0 (or a read-time finalisation)
    // sums once this kernel has ended
    __syncthreads();
    if (threadIdx.x == 0) {
        // one acquire-release add: releases this block's writes (ordered
        // before it by the barrier), and the last block acquires the others'
        s_last = atom_add_acq_rel_gpu(P.fin_count, 1u) == gridDim.x - 1;
        if (s_last) {
            if (__ldcg(&st->err)) {   // a failed step is not published
                *P.fin_count = 0;
            } else {
                st->rho_nblk = gridDim.x;
                st->rho_pending = tn;
                publish_step(P, st, tn, MM, step_counts(P, st, tn));
            }
        }
    }
    if constexpr (BATCH) {   // this block's sums per instance (complete: the loop ended with a barrier)
        double2 *part = rho_part_of(P, tn, MM) + (size_t)blockIdx.x * P.n_inst * (MM + 1);
        for (int i = threadIdx.x; i < P.n_inst * (MM + 1); i += NT) part[i] = s_acc[i];
        return;
    }
    // this block's partials of rho(t+1) and survivor count; a block that
    // processed no tile writes zeros without reducing (s_any: thread 0 holds
    // block_kept; the barrier below orders it)
    float4 *mine = spart_of(P, tn, MM) + (size_t)blockIdx.x * MM;
    if constexpr (kTileAccS) {   // the warps' pairs merged in order (thread k: end point k; zeros without a tile)
        if ((int)threadIdx.x < MM) {
            const int k = threadIdx.x;
            float4 a = s_wrho[0][k];
            for (int w = 1; w < NW; ++w) {
                const float4 b = s_wrho[w][k];
                const float tx = a.x + b.x, vx = tx - a.x;
                a.y += b.y + ((a.x - (tx - vx)) + (b.x - vx));
                a.x = tx;
                const float ty = a.z + b.z, vy = ty - a.z;
                a.w += b.w + ((a.z - (ty - vy)) + (b.z - vy));
                a.z = ty;
            }
            mine[k] = a;
        }
    } else {
        if (threadIdx.x == 0) s_any = block_kept > 0 || s_any;
        __syncthreads();
        if (s_any) {
            float2 lo[MM];
#pragma unroll
            for (int k = 0; k < MM; ++k) {
                if constexpr (kKahan) lo[k] = make_float2(-rcmp[k].x, -rcmp[k].y);
                else lo[k] = make_float2(0.f, 0.f);
            }
            block_rho_pair<MM, NW, C64>(racc, lo, s_rt, mine);
        } else if ((int)threadIdx.x < MM) {
            mine[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (threadIdx.x == 0) scount_of(P, tn)[blockIdx.x] = (long long)block_kept;
}

template <int M, bool C64, int NX, int S>
__global__ void __launch_bounds__(kStreamThreads, (M == 2 || (M == 3 && C64)) ? 2 : 1)
    k_stream_step(Params P, int lut_smem) {
    stream_step_body<M, C64, NX, S, false>(P, lut_smem);
}

// Batched stream engine: nsteps steps of all instances, separated by
// bounded grid barriers (a cooperative launch when nsteps > 1; one step is
// an ordinary launch).  The stored set lives in n_inst * M*M regions
// (instance, newest point); tickets run over the tiles of all regions in
// order, so an instance's tiles are consecutive and its look-back stops at
// its first tile.
template <int M, bool C64, int S>
__global__ void __launch_bounds__(kStreamThreads, (M == 2 || (M == 3 && C64)) ? 2 : 1)
    k_stream_batch(Params P, int nsteps) {
    for (int s = 0; s < nsteps; ++s) {
        stream_step_body<M, C64, 1, S, true>(P, 0);
        if (s + 1 < nsteps && grid_barrier(P.st)) break;
    }
}

// The kernels' FP32 -> FP64 widening over an array (test hook).
__global__ void k_widen(const float *in, double *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = f2d_exact(in[i]);
}

// ---------------------------------------------------------------- post-merging engine
//
// The original order of the method (Sec. 2.1, Scheme macgic: propagation(),
// sorting(), merging()), for the comparison the paper makes with the
// pre-merging order (Sec. 4.1).  Per step: every stored path is extended by
// its M^2 children with its own history (phase_expand without a merge), the
// survivors of the filter go to the unmerged buffer (Omega(t, unmerged)) and
// rho(t) is summed from them; the children are then sorted by their masked
// key (the mask P itself; while the window fills, the whole key, so nothing
// merges) with a stable least-significant-digit radix sort of 8-bit digits
// over (key, child index) pairs, and every run of equal masked keys becomes
// one stored path: the child of largest weight (R4) with the run's sum.

constexpr int kSortThreads = 256;                      // = number of digit values
constexpr int kSortIpt = 16;                           // items per thread of a sort chunk
constexpr int kSortChunk = kSortThreads * kSortIpt;    // 4096 items per chunk
constexpr int kScanThreads = 1024;
constexpr int kScanSeg = 4 * kScanThreads;             // elements per block of the multi-block scan

__device__ __forceinline__ long long post_chunks(const DevState *st) {
    return (long long)((st->post_n + kSortChunk - 1) / kSortChunk);
}
// Length of the array a multi-block scan runs over: the digit counts of a
// radix pass (which = 0) or the run heads per chunk (which = 1).
__device__ __forceinline__ long long scan_len(const DevState *st, int which) {
    const long long nch = post_chunks(st);
    return which == 0 ? 256 * nch : nch;
}
// A radix pass is active while its digit lies inside the step's key bits.
__device__ __forceinline__ bool pass_active(const DevState *st, int pass) {
    return 8 * pass < (int)st->post_bits;
}

// Masked key compressed to consecutive bits: the runs of consecutive mask
// positions packed one after another.
__device__ __forceinline__ unsigned long long compress_masked(const Params &P, unsigned long long key) {
    unsigned long long c = 0;
    for (int r = 0; r < P.nruns; ++r) c |= ((key >> P.run_shift[r]) & P.run_mask[r]) << P.run_off[r];
    return c;
}

template <int M, bool C64>
__global__ void __launch_bounds__(kExpandThreads) k_post_expand(Params P) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    phase_expand<M, C64, kExpandThreads, false>(P, t, st->n_cur, false, &st->cnt_out[tn % 3], rho_part_of(P, tn, M * M),
                                                P.ckeys, P.camps);
}

// Sort keys of the unmerged children: the masked key compressed once the
// children's window is full, the whole key before (nothing merges then).
__global__ void k_post_keys(Params P) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long tn = st->t + 1;
    const unsigned long long n = __ldcg(&st->cnt_out[tn % 3]);
    const bool full = tn + 1 >= (unsigned long long)P.dkmax;
    const int L_child = (int)min(tn + 1, (unsigned long long)P.dkmax);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->post_n = n;
        st->post_bits = full ? (unsigned)P.post_bits_full : (unsigned)(P.b * L_child);
    }
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long k = __ldcg(P.ckeys + i);
        P.skey[0][i] = full ? (P.post_compress ? compress_masked(P, k) : (k & P.pmask)) : k;
        P.sidx[0][i] = (unsigned)i;
    }
}

// Radix pass, step 1: digit counts per chunk, stored digit-major
// (rs_hist[d * chunks + c]) so that one exclusive scan of the whole array
// gives every (digit, chunk) its first output position.
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(Params P, int pass) {
    DevState *st = P.st;
    if (st->err || !pass_active(st, pass)) return;
    const unsigned long long n = st->post_n;
    const long long nch = post_chunks(st);
    const int shift = 8 * pass;
    const unsigned long long *in = P.skey[pass & 1];
    __shared__ unsigned h[256];
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const unsigned long long b0 = (unsigned long long)c * kSortChunk;
        for (int j = threadIdx.x; j < kSortChunk; j += kSortThreads) {
            const unsigned long long i = b0 + j;
            if (i < n) atomicAdd(&h[(unsigned)(__ldcg(in + i) >> shift) & 255u], 1u);
        }
        __syncthreads();
        P.rs_hist[(size_t)threadIdx.x * nch + c] = h[threadIdx.x];
        __syncthreads();
    }
}

// Exclusive scan of a block's kScanThreads * 4 elements held 4 per thread
// (v[0..3], consecutive); returns the thread's exclusive prefix and the
// block total in *tot.  All threads call it.
__device__ __forceinline__ unsigned block_scan4(const unsigned v[4], unsigned *tot) {
    __shared__ unsigned s_w[kScanThreads / 32];
    __shared__ unsigned s_tot;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned mine = v[0] + v[1] + v[2] + v[3];
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned x = lane < kScanThreads / 32 ? s_w[lane] : 0u;
        unsigned xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, xi, o);
            if ((int)lane >= o) xi += y;
        }
        if (lane < kScanThreads / 32) s_w[lane] = xi - x;
        if (lane == 31) s_tot = xi;
    }
    __syncthreads();
    const unsigned r = s_w[warp] + incl - mine;
    *tot = s_tot;
    __syncthreads();
    return r;
}

// Exclusive scan of one value per thread over a block of NT threads (all
// threads call it).
template <int NT>
__device__ __forceinline__ unsigned block_excl_scan(unsigned v) {
    __shared__ unsigned s_w[NT / 32];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned a = 0;
        for (int w = 0; w < NT / 32; ++w) {
            const unsigned x = s_w[w];
            s_w[w] = a;
            a += x;
        }
    }
    __syncthreads();
    const unsigned r = s_w[warp] + incl - v;
    __syncthreads();
    return r;
}

// Multi-block exclusive scan, in place (three kernels): block partials,
// their scan (one block; it also stores the total), and the blocks' own
// scans from their bases.
__global__ void __launch_bounds__(kScanThreads) k_scan_part(Params P, unsigned *a, int which, int pass) {
    DevState *st = P.st;
    if (st->err || (which == 0 && !pass_active(st, pass))) return;
    const long long len = scan_len(st, which);
    const long long nb = (len + kScanSeg - 1) / kScanSeg;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        unsigned v[4];
        for (int u = 0; u < 4; ++u) {
            const long long i = b * kScanSeg + 4 * (long long)threadIdx.x + u;
            v[u] = i < len ? a[i] : 0u;
        }
        unsigned tot;
        block_scan4(v, &tot);
        if (threadIdx.x == 0) P.rs_part[b] = tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(Params P, int which, int pass) {
    DevState *st = P.st;
    if (st->err || (which == 0 && !pass_active(st, pass))) return;
    const long long len = scan_len(st, which);
    const long long nb = (len + kScanSeg - 1) / kScanSeg;
    unsigned long long carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += kScanSeg) {
        unsigned v[4];
        for (int u = 0; u < 4; ++u) {
            const long long i = b0 + 4 * (long long)threadIdx.x + u;
            v[u] = i < nb ? P.rs_part[i] : 0u;
        }
        unsigned tot;
        const unsigned ex = block_scan4(v, &tot);
        unsigned run = ex;
        for (int u = 0; u < 4; ++u) {
            const long long i = b0 + 4 * (long long)threadIdx.x + u;
            if (i < nb) P.rs_part[i] = (unsigned)(carry + run);
            run += v[u];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) st->scan_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(Params P, unsigned *a, int which, int pass) {
    DevState *st = P.st;
    if (st->err || (which == 0 && !pass_active(st, pass))) return;
    const long long len = scan_len(st, which);
    const long long nb = (len + kScanSeg - 1) / kScanSeg;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        unsigned v[4];
        for (int u = 0; u < 4; ++u) {
            const long long i = b * kScanSeg + 4 * (long long)threadIdx.x + u;
            v[u] = i < len ? a[i] : 0u;
        }
        unsigned tot;
        unsigned run = P.rs_part[b] + block_scan4(v, &tot);
        for (int u = 0; u < 4; ++u) {
            const long long i = b * kScanSeg + 4 * (long long)threadIdx.x + u;
            if (i < len) a[i] = run;
            run += v[u];
        }
    }
}

// Radix pass, step 3: stable scatter.  Warp w of a chunk owns the items
// [w SC, (w+1) SC) and visits them 32 at a time in order; lanes with equal
// digits find each other with a match and rank among themselves, the warp's
// running count per digit orders its rounds, and the warps' counts (scanned
// across warps) order the warps: the output keeps the input order among
// equal digits.
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(Params P, int pass) {
    DevState *st = P.st;
    if (st->err || !pass_active(st, pass)) return;
    constexpr int NW = kSortThreads / 32, SC = kSortChunk / NW, IT = SC / 32;
    const unsigned long long n = st->post_n;
    const long long nch = post_chunks(st);
    const int shift = 8 * pass;
    const unsigned long long *ik = P.skey[pass & 1];
    const unsigned *ii = P.sidx[pass & 1];
    unsigned long long *ok = P.skey[(pass + 1) & 1];
    unsigned *oi = P.sidx[(pass + 1) & 1];
    __shared__ unsigned s_wc[NW][256];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        for (int w = 0; w < NW; ++w) s_wc[w][threadIdx.x] = 0u;
        __syncthreads();
        const unsigned long long base = (unsigned long long)c * kSortChunk + (unsigned long long)warp * SC;
        unsigned long long kk[IT];
        unsigned xx[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const unsigned long long i = base + (unsigned long long)it * 32 + lane;
            const bool valid = i < n;
            kk[it] = valid ? __ldcg(ik + i) : 0ull;
            xx[it] = valid ? __ldcg(ii + i) : 0u;
            const unsigned d = valid ? ((unsigned)(kk[it] >> shift) & 255u) : 256u + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid && (peers & lt) == 0u) s_wc[warp][d] += (unsigned)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // first output position of each (warp, digit): chunk base of the digit + earlier warps
            const int d = threadIdx.x;
            unsigned acc = P.rs_hist[(size_t)d * nch + c];
            for (int w = 0; w < NW; ++w) {
                const unsigned v = s_wc[w][d];
                s_wc[w][d] = acc;
                acc += v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const unsigned long long i = base + (unsigned long long)it * 32 + lane;
            const bool valid = i < n;
            const unsigned d = valid ? ((unsigned)(kk[it] >> shift) & 255u) : 256u + lane;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (valid) {
                const unsigned pos = s_wc[warp][d] + (unsigned)__popc(peers & lt);
                ok[pos] = kk[it];
                oi[pos] = xx[it];
            }
            __syncwarp();
            if (valid && (peers & lt) == 0u) s_wc[warp][d] += (unsigned)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
    }
}

// Sorted keys of the step: the buffer the last active pass wrote.
__device__ __forceinline__ int sorted_buf(const DevState *st) { return (int)(((st->post_bits + 7u) / 8u) & 1u); }

// Reduce by key, step 1: run heads per chunk of the sorted keys.
__global__ void __launch_bounds__(kSortThreads) k_rbk_heads(Params P) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long n = st->post_n;
    const long long nch = post_chunks(st);
    const unsigned long long *sk = P.skey[sorted_buf(st)];
    __shared__ unsigned s_n;
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        unsigned cnt = 0;
        for (int j = threadIdx.x; j < kSortChunk; j += kSortThreads) {
            const unsigned long long i = (unsigned long long)c * kSortChunk + j;
            if (i < n && (i == 0 || __ldcg(sk + i) != __ldcg(sk + i - 1))) ++cnt;
        }
        atomicAdd(&s_n, cnt);
        __syncthreads();
        if (threadIdx.x == 0) P.rbk_heads[c] = s_n;
        __syncthreads();
    }
}

// Reduce by key, step 2: each run head's thread walks its run (in sorted
// order, which is the unmerged buffer's order among equal keys): the sum
// (C64: FP32 with every rounding error kept, rounded once; FP64: FP64), the
// largest weight, then the smallest full key within the tie window (R4);
// the run becomes one stored path of Omega(t) at the position of its head
// among all heads.
template <bool C64>
__global__ void __launch_bounds__(kSortThreads) k_rbk_write(Params P) {
    using AmpT = typename std::conditional<C64, float2, double2>::type;
    using WT = typename std::conditional<C64, float, double>::type;
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long tn = st->t + 1;
    const unsigned long long n = st->post_n;
    const long long nch = post_chunks(st);
    const int sb = sorted_buf(st);
    const unsigned long long *sk = P.skey[sb];
    const unsigned *si = P.sidx[sb];
    const AmpT *camps = static_cast<const AmpT *>(P.camps);
    unsigned long long *keys_out = P.keys[tn & 1];
    AmpT *amps_out = static_cast<AmpT *>(P.amps[tn & 1]);
    const WT tie = (WT)(1.0 - P.tie_rel);
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        // this thread's kSortIpt consecutive items of the chunk
        const unsigned long long i0 = (unsigned long long)c * kSortChunk + (unsigned long long)threadIdx.x * kSortIpt;
        unsigned hm = 0;
        for (int u = 0; u < kSortIpt; ++u) {
            const unsigned long long i = i0 + u;
            if (i < n && (i == 0 || __ldcg(sk + i) != __ldcg(sk + i - 1))) hm |= 1u << u;
        }
        unsigned pos = P.rbk_heads[c] + block_excl_scan<kSortThreads>((unsigned)__popc(hm));
        for (unsigned m = hm; m; m &= m - 1u) {
            const unsigned long long h = i0 + (__ffs(m) - 1);
            const unsigned long long mk = __ldcg(sk + h);
            float sx = 0.f, sy = 0.f, ex = 0.f, ey = 0.f;
            double dx = 0.0, dy = 0.0;
            WT wmax = 0;
            unsigned long long j = h;
            for (; j < n && __ldcg(sk + j) == mk; ++j) {
                const AmpT a = camps[__ldcg(si + j)];
                if constexpr (C64) {
                    two_sum_acc(sx, ex, a.x);
                    two_sum_acc(sy, ey, a.y);
                } else {
                    dx += a.x;
                    dy += a.y;
                }
                const WT w2 = a.x * a.x + a.y * a.y;
                wmax = w2 > wmax ? w2 : wmax;
            }
            unsigned long long rep = kEmpty;
            for (unsigned long long k = h; k < j; ++k) {
                const unsigned x = __ldcg(si + k);
                const AmpT a = camps[x];
                const WT w2 = a.x * a.x + a.y * a.y;
                const unsigned long long key = P.ckeys[x];
                if (w2 >= tie * wmax && key < rep) rep = key;
            }
            keys_out[pos] = rep;
            if constexpr (C64) amps_out[pos] = make_float2(sx + ex, sy + ey);
            else amps_out[pos] = make_double2(dx, dy);
            ++pos;
        }
    }
}

// Publishes a post-merging step: rho(t) from the extension's block partials,
// the merged count, the statistics (intermediate = the unmerged children).
__global__ void __launch_bounds__(256) k_post_publish(Params P, int MM, int nblk) {
    DevState *st = P.st;
    if (st->err) return;
    const unsigned long long t = st->t, tn = t + 1;
    phase_finalize(P, tn, 0, rho_part_of(P, tn, MM), nblk, MM);
    if (threadIdx.x != 0) return;
    const unsigned long long n_in = st->n_cur, inter = st->post_n, merged = st->scan_total;
    StepRec r;
    r.t = (long long)tn;
    r.groups = (long long)n_in;
    r.extended = (long long)n_in * MM;
    r.kept = (long long)merged;
    r.inter = (long long)inter;
    const size_t slot = (size_t)(tn % (unsigned long long)P.rho_hist);
    P.stats_ring[slot] = r;
    P.inst_kept[slot] = (long long)merged;
    st->n_cur = merged;
    st->t = tn;
    st->cnt_groups[(tn + 1) % 3] = 0;
    st->cnt_out[(tn + 1) % 3] = 0;
}

// ---------------------------------------------------------------- ranks
//
// Sharded propagation over several GPUs (the distributed pre-merge of Sec.
// 3.2, in a GPU form: owner routing instead of the sequential broadcast
// rounds).  Every stored path belongs to the rank that owns its next
// pre-merge group, so that each rank's groups are complete:
//   owner = ((key & P'-bits) * 0x9E3779B97F4A7C15 >> 32) mod n_ranks.
// k_part_count counts the stored paths per owner, k_part_scatter copies
// them grouped by owner (rank 0's first) into the caller's buffers.

constexpr int kMaxRanks = 1024;

__device__ __forceinline__ unsigned owner_rank(const Params &P, unsigned long long key, unsigned n_ranks) {
    const unsigned long long h = ((key & P.pmask) * 0x9E3779B97F4A7C15ull) >> 32;
    return (unsigned)(h % n_ranks);
}

__global__ void k_part_count(Params P, unsigned n_ranks, unsigned long long *cnt) {
    __shared__ unsigned s_c[kMaxRanks];
    const DevState *st = P.st;
    const unsigned long long n = st->n_cur;
    const unsigned long long *keys = P.keys[st->t & 1];
    for (unsigned r = threadIdx.x; r < n_ranks; r += blockDim.x) s_c[r] = 0;
    __syncthreads();
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        atomicAdd(&s_c[owner_rank(P, keys[i], n_ranks)], 1u);
    __syncthreads();
    for (unsigned r = threadIdx.x; r < n_ranks; r += blockDim.x)
        if (s_c[r]) atomicAdd(&cnt[r], (unsigned long long)s_c[r]);
}

template <typename Amp>
__global__ void k_part_scatter(Params P, unsigned n_ranks, const unsigned long long *base, unsigned long long *cursor,
                               unsigned long long *keys_out, Amp *amps_out) {
    const DevState *st = P.st;
    const unsigned long long n = st->n_cur;
    const unsigned long long *keys = P.keys[st->t & 1];
    const Amp *amps = static_cast<const Amp *>(P.amps[st->t & 1]);
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const unsigned r = owner_rank(P, k, n_ranks);
        const unsigned long long o = base[r] + atomicAdd(&cursor[r], 1ull);
        keys_out[o] = k;
        amps_out[o] = amps[i];
    }
}

// Sets the stored count after an import (one thread).
__global__ void k_set_count(DevState *st, unsigned long long n) { st->n_cur = n; }

// ---------------------------------------------------------------- set-up kernels

__global__ void k_clear_table(Slot *slots, unsigned long long *repk, unsigned long long n) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        Slot s;
        s.mk = kEmpty;
        s.wmax = 0ull;
        s.sre = 0.0;
        s.sim = 0.0;
        slots[i] = s;
        repk[i] = kEmpty;
    }
}

// History tables: for n_act = 1..dkmax, chunk j (one byte of the key), byte
// value v: sum over the positions p of the byte with p <= n_act - 2 of
// eta_{p+1} q[s+_p] - conj(eta_{p+1}) q[s-_p] (lag p+1 of the new point).
// eta0 (symmetric splitting, else NULL): while the window fills (n_act <
// dkmax) the oldest position n_act - 1 holds point 0, which enters with its
// own coefficient eta0[n_act] (its half interval) instead of being left out.
__global__ void k_build_lut(double2 *lut, float2 *lutf, float2 *lutlo, const double2 *eta, const double *q,
                            int M, int bs, int b, int dkmax, int nchunks, const double2 *eta0) {
    const int total = dkmax * nchunks * kLutEntries;
    const int ppc = 8 / b;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int v = i % kLutEntries;
        const int j = (i / kLutEntries) % nchunks;
        const int n_act = i / (kLutEntries * nchunks) + 1;
        double hx = 0.0, hy = 0.0;
        for (int k = 0; k < ppc; ++k) {
            const int p = j * ppc + k;
            const bool point0 = eta0 != nullptr && n_act < dkmax && p == n_act - 1;
            if (p > n_act - 2 && !point0) continue;
            const int code = (v >> (b * k)) & ((1 << b) - 1);
            const int sp = code & ((1 << bs) - 1), sm = code >> bs;
            if (sp >= M || sm >= M) continue;   // codes that never occur
            const double2 e = point0 ? eta0[n_act] : eta[p + 1];
            // eta q+ - conj(eta) q-
            hx += e.x * q[sp] - e.x * q[sm];
            hy += e.y * q[sp] + e.y * q[sm];
        }
        lut[i] = make_double2(hx, hy);
        const float fx = (float)hx, fy = (float)hy;
        lutf[i] = make_float2(fx, fy);
        lutlo[i] = make_float2((float)(hx - (double)fx), (float)(hy - (double)fy));
    }
}

// W[(a,b)][(a',b')] = U[a,a'] conj(U[b,b']) exp(-(q_a - q_b)(eta_0 q_a - conj(eta_0) q_b))
__global__ void k_build_w(double2 *w, float4 *wf, const double2 *U, const double2 *eta, const double *q, int M) {
    const int MM = M * M;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MM * MM; i += gridDim.x * blockDim.x) {
        const int child = i / MM, par = i % MM;
        const int a = child / M, b = child % M, ap = par / M, bp = par % M;
        const double2 ua = U[a * M + ap];
        const double2 ub = U[b * M + bp];
        const double2 prop = make_double2(ua.x * ub.x + ua.y * ub.y, ua.y * ub.x - ua.x * ub.y);  // ua * conj(ub)
        const double dq = q[a] - q[b];
        const double2 e0 = eta[0];
        // z = -(dq) (e0 q_a - conj(e0) q_b)
        const double inner_x = e0.x * q[a] - e0.x * q[b];
        const double inner_y = e0.y * q[a] + e0.y * q[b];
        const double zr = -dq * inner_x, zi = -dq * inner_y;
        double s, c;
        sincos(zi, &s, &c);
        const double m = exp(zr);
        const double2 wv = cmul(prop, make_double2(m * c, m * s));
        w[i] = wv;
        const float hx = (float)wv.x, hy = (float)wv.y;
        wf[i] = make_float4(hx, hy, (float)(wv.x - (double)hx), (float)(wv.y - (double)hy));
    }
}

// exp(-delta_d T) for every history table entry T[n_act][j][v] and every
// distinct nonzero coupling difference delta_d (FP64 extension path).
__global__ void k_build_etab(double2 *etab, const double2 *lut, const double *deltas, int ndelta, int dkmax,
                             int nchunks) {
    const long long per = (long long)nchunks * kLutEntries;
    const long long total = (long long)dkmax * ndelta * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i % per;
        const int d = (int)((i / per) % ndelta);
        const int n = (int)(i / (per * ndelta));
        const double2 T = lut[(long long)n * per + r];
        const double zr = -deltas[d] * T.x, zi = -deltas[d] * T.y;
        double sn, cs;
        sincos(zi, &sn, &cs);
        const double m = exp(zr);
        etab[i] = make_double2(m * cs, m * sn);
    }
}

// ---------------------------------------------------------------- host side

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
    size_t keys[2], amps[2], slots, repk, slot_of, groups, lut, lutf, lutlo, etab, wtab, wtabf, uprop, eta, q, deltas,
        rho, rho_part, spart, scount, stats, inst_kept, fin_count, tile_state, reg_n, state, total;
    size_t ckeys, camps, skey[2], sidx[2], rs_hist, rs_part, rbk_heads;   // post-merging engine
    size_t ranks;                                                        // per-rank counts, bases, cursors
    size_t lutE, lutEf, lutElo, etabE, wEt, wEtf, eta0d, dEd, dE0d;       // symmetric splitting
    long long max_chunks;
    long long entries, max_tiles;
    size_t nlut;           // history-table entries of one instance
    int nd;                // distinct nonzero coupling differences
    unsigned long long tcap;
    unsigned int tcap_log2;
    int nchunks;
};

int bits_per_state(int M) {
    int bs = 1;
    while ((1 << bs) < M) ++bs;
    return bs;
}

int inst_bits(int n_inst) {
    int ib = 0;
    while ((1 << ib) < n_inst) ++ib;
    return ib;
}

const char *validate(const qp_config *c) {
    if (!c) return "null config";
    if (c->M < 2 || c->M > 4) return "M must be 2..4";
    if (c->dkmax < 1) return "dkmax must be >= 1";
    const int b = 2 * bits_per_state(c->M);
    if (b * c->dkmax > 64) return "b*dkmax exceeds the 64-bit key";
    if (!(c->dt > 0.0) || !std::isfinite(c->dt)) return "dt must be positive";
    if (!c->q || !c->hs_re) return "q and hs_re are required";
    if (c->precision != QP_FP64 && c->precision != QP_C64) return "unknown precision";
    if (c->engine < QP_ENGINE_AUTO || c->engine > QP_ENGINE_STREAM) return "unknown engine";
    if (!(c->theta >= 0.0) || !std::isfinite(c->theta)) return "theta must be >= 0";
    if (c->max_paths < 1 || c->max_paths > (int64_t(1) << 40)) return "max_paths out of range";
    if (c->max_groups < 0 || c->max_groups > (int64_t(1) << 30)) return "max_groups out of range";
    if (c->engine != QP_ENGINE_STREAM && c->max_groups == 0 && c->max_paths > (int64_t(1) << 30))
        return "set max_groups (<= 2^30) for max_paths > 2^30 (the merge table; not needed by the stream engine)";
    if (c->rho_history < 0 || c->rho_history > (1 << 24)) return "rho_history out of range";
    if (c->n_inst < 0 || c->n_inst > kMaxInst) return "n_inst out of range (0..128)";
    if (c->scheme != QP_PREMERGE && c->scheme != QP_POSTMERGE) return "unknown scheme";
    if (c->scheme == QP_POSTMERGE && c->n_inst > 1) return "the post-merging scheme takes single problems only";
    if (c->scheme == QP_POSTMERGE && c->max_paths > (int64_t(1) << 32) - 1)
        return "post-merging: max_paths (the unmerged set) must stay below 2^32";
    if (b * c->dkmax + inst_bits(c->n_inst) > 64) return "b*dkmax plus the instance index exceed the 64-bit key";
    for (int i = 0; i < c->M; ++i)
        if (!std::isfinite(c->q[i])) return "q must be finite";
    for (int i = 0; i < c->M * c->M; ++i) {
        const int r = i / c->M, k = i % c->M;
        const double im = c->hs_im ? c->hs_im[i] : 0.0, imT = c->hs_im ? c->hs_im[k * c->M + r] : 0.0;
        if (!std::isfinite(c->hs_re[i]) || !std::isfinite(im)) return "H_S must be finite";
        if (std::fabs(c->hs_re[i] - c->hs_re[k * c->M + r]) > 1e-12 || std::fabs(im + imT) > 1e-12)
            return "H_S must be Hermitian";
    }
    return nullptr;
}

// Distinct nonzero differences q_a - q_b (a != b); dsel[a*M+b] = index or -1.
int distinct_deltas(int M, const double *q, std::vector<double> *vals, signed char *dsel) {
    std::vector<double> v;
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
            const double d = q[a] - q[b];
            int idx = -1;
            if (d != 0.0) {
                for (size_t k = 0; k < v.size(); ++k)
                    if (v[k] == d) idx = (int)k;
                if (idx < 0) {
                    v.push_back(d);
                    idx = (int)v.size() - 1;
                }
            }
            if (dsel) dsel[a * M + b] = (signed char)idx;
        }
    if (vals) *vals = v;
    return (int)v.size();
}

// Equally spaced coupling eigenvalues q_a = q_0 + a s (s != 0, exact in
// FP64): the children's influence factors are powers of exp(-s H).  Sets
// P.qeq and the indices of +s and -s among the distinct differences.
void set_equispaced(Params &P, int M, const double *q, const double *deltas, int nd) {
    P.qeq = 0;
    P.d_pos = P.d_neg = 0;
    P.qstepf = 0.f;
    const double s = q[1] - q[0];
    if (s == 0.0) return;
    for (int a = 0; a < M; ++a)
        if (q[a] - q[0] != (double)a * s) return;
    int ip = -1, in = -1;
    for (int k = 0; k < nd; ++k) {
        if (deltas[k] == s) ip = k;
        if (deltas[k] == -s) in = k;
    }
    if (ip < 0 || in < 0) return;
    P.qeq = 1;
    P.d_pos = ip;
    P.d_neg = in;
    P.qstepf = (float)s;
}

Layout make_layout(const qp_config *c) {
    Layout L{};
    const long long mp = c->max_paths;
    // the stream engine, when asked for explicitly, never uses the merge
    // table or the group arrays: they shrink to a token size, leaving the
    // memory to the path buffers (about 2 * (8 + amplitude) bytes per path)
    const bool stream_only = c->engine == QP_ENGINE_STREAM;
    const long long mg = stream_only ? 1 : (c->max_groups ? c->max_groups : c->max_paths);
    const size_t ampb = c->precision == QP_C64 ? sizeof(float2) : sizeof(double2);
    unsigned int lg = 4;
    while ((1ull << lg) < 2ull * (unsigned long long)mg) ++lg;
    L.tcap = 1ull << lg;
    L.tcap_log2 = lg;
    const int b = 2 * bits_per_state(c->M);
    L.nchunks = (c->dkmax - 1) * b > 0 ? ((c->dkmax - 1) * b + 7) / 8 : 0;
    const int R = c->rho_history ? c->rho_history : 4096;
    const int MM = c->M * c->M;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.state = take(sizeof(DevState));
    // path buffers: a flat array of max_paths entries (merge-table engine),
    // or the same memory as M*M regions of max_paths / (M*M) (stream engine)
    const long long ent = mp;
    L.entries = ent;
    L.keys[0] = take(ent * 8);
    L.keys[1] = take(ent * 8);
    L.amps[0] = take(ent * ampb);
    L.amps[1] = take(ent * ampb);
    L.slots = take(L.tcap * sizeof(Slot));
    L.repk = take(L.tcap * 8);
    L.slot_of = take(stream_only ? 4 : mp * 4);
    L.groups = take(mg * 4);
    const int NI = std::max(1, c->n_inst);
    const size_t nlut = (size_t)c->dkmax * std::max(1, L.nchunks) * kLutEntries;
    L.nlut = nlut;
    L.lut = take(NI * nlut * sizeof(double2));
    L.lutf = take(NI * nlut * sizeof(float2));
    L.lutlo = take(NI * nlut * sizeof(float2));
    const int nd = distinct_deltas(c->M, c->q, nullptr, nullptr);
    L.nd = nd;
    L.etab = take(NI * nlut * std::max(1, nd) * sizeof(double2));
    L.wtab = take((size_t)NI * MM * MM * sizeof(double2));
    L.wtabf = take((size_t)NI * MM * MM * sizeof(float4));
    L.deltas = take(kMaxDelta * sizeof(double));
    L.uprop = take(MM * sizeof(double2));
    L.eta = take((size_t)NI * c->dkmax * sizeof(double2));
    L.q = take(c->M * sizeof(double));
    L.rho = take((size_t)R * NI * MM * sizeof(double2));
    L.rho_part = take((size_t)2 * kMaxExpandBlocks * NI * (MM + 1) * sizeof(double2));   // by step parity
    L.spart = take((size_t)2 * kMaxExpandBlocks * MM * sizeof(float4));
    L.scount = take((size_t)2 * kMaxExpandBlocks * sizeof(long long));
    L.stats = take((size_t)R * sizeof(StepRec));
    L.inst_kept = take((size_t)R * NI * sizeof(long long));
    L.fin_count = take(sizeof(unsigned int));
    // stream regions: one per (instance, newest point); at the smallest tile
    // every region may end in a partial tile
    const long long nreg = (long long)NI * MM;
    L.max_tiles = nreg * ((mp / nreg + kStreamMinTile - 1) / kStreamMinTile + 1);
    L.tile_state = take((size_t)L.max_tiles * MM * 8);
    L.reg_n = take((size_t)2 * nreg * 8);
    L.ranks = take((size_t)3 * kMaxRanks * 8);
    if (NI == 1) {   // symmetric splitting (single problems): correction tables, coefficient arrays
        L.lutE = take(nlut * sizeof(double2));
        L.lutEf = take(nlut * sizeof(float2));
        L.lutElo = take(nlut * sizeof(float2));
        L.etabE = take(nlut * std::max(1, nd) * sizeof(double2));
        L.wEt = take((size_t)MM * MM * sizeof(double2));
        L.wEtf = take((size_t)MM * MM * sizeof(float4));
        L.eta0d = take((size_t)c->dkmax * sizeof(double2));
        L.dEd = take((size_t)c->dkmax * sizeof(double2));
        L.dE0d = take((size_t)c->dkmax * sizeof(double2));
    }
    if (c->scheme == QP_POSTMERGE) {   // unmerged set, sort pairs, digit counts, scan partials, run heads
        L.max_chunks = (mp + kSortChunk - 1) / kSortChunk + 1;
        L.ckeys = take(mp * 8);
        L.camps = take(mp * ampb);
        for (int k = 0; k < 2; ++k) {
            L.skey[k] = take(mp * 8);
            L.sidx[k] = take(mp * 4);
        }
        L.rs_hist = take((size_t)256 * L.max_chunks * 4);
        L.rs_part = take(((size_t)256 * L.max_chunks / kScanSeg + 2) * 4);
        L.rbk_heads = take((size_t)L.max_chunks * 4);
    }
    L.total = off;
    return L;
}

}  // namespace

struct qp_ctx {
    qp_config cfg;
    std::vector<double> q;
    std::vector<qp::cplx> hs, U;
    std::vector<double> deltas;
    Layout L;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    int device = 0, nsm = 0;
    Params P{};
    bool have_eta = false, have_state = false, failed = false;
    std::vector<int> mask;
    int persist_grid = 0;              // blocks of the cooperative persistent kernel (0 = not usable)
    int persist_max = 0;               // co-resident limit of that kernel
    bool use_persistent = true;
    int bps_ins = 4, bps_exp = 4;      // blocks per SM of the pre-merge and extension kernels
    int graph_steps = 1;               // steps captured per CUDA graph
    int stream_nx = 0;                 // stream engine usable with the mask: sub-groups per run (0 = no)
    int stream_tile = 1024;            // stored paths per tile of the stream engine
    const void *scache_fn = nullptr;   // stream kernel launched last, its dynamic shared memory and
    size_t scache_smem = 0;            // co-resident blocks per SM
    int scache_res = 0;
    const void *rcache_fn = nullptr;   // the same for the regular stream kernel
    size_t rcache_smem = 0;
    int rcache_res = 0;
    bool use_stream = false;           // this propagation runs on the stream engine
    bool sym = false;                  // symmetric Trotter splitting (qp_set_end_points)
    qp::cplx eta00;                    // ... point 0's half-interval self coefficient
    cudaGraphExec_t graph1 = nullptr;  // one-step graph for remainders
    cudaGraphExec_t graph = nullptr;
    bool graph_dirty = true;
    bool use_graph = true;
    int64_t host_t = 0;                // steps enqueued since qp_set_rho0 (set from the device at every state read)
    void *hpin = nullptr;              // pinned host staging for rho reads (state + rows)
    size_t hpin_bytes = 0;
    std::string err;
};

namespace {

qp_status fail(qp_ctx *c, qp_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

#define QP_CUDA(ctx, call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(ctx, QP_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kStepKernels = 4;

// Launch one step; if ev is given, record ev[k] before kernel k and
// ev[kStepKernels] after the last one.
size_t batch_smem(const qp_ctx *c) {
    const int MM = c->cfg.M * c->cfg.M;
    return c->P.n_inst > 1 ? (size_t)c->P.n_inst * (MM + 1) * sizeof(double2) : 0;
}

template <int M, typename Amp>
cudaError_t launch_step_t(qp_ctx *c, cudaEvent_t *ev) {
    constexpr bool C64 = sizeof(Amp) == sizeof(float2);
    const int g_ins = c->nsm * c->bps_ins;
    const int g_exp = std::min(c->nsm * c->bps_exp, kMaxExpandBlocks);
    const size_t sm = batch_smem(c);
    if (ev) cudaEventRecord(ev[0], c->stream);
    k_insert<Amp><<<g_ins, kInsertThreads, 0, c->stream>>>(c->P);
    if (ev) cudaEventRecord(ev[1], c->stream);
    k_tiebreak<Amp><<<g_ins, kInsertThreads, 0, c->stream>>>(c->P);
    if (ev) cudaEventRecord(ev[2], c->stream);
    if (c->P.n_inst > 1)
        k_expand<M, C64, true><<<g_exp, kExpandThreads, sm, c->stream>>>(c->P);
    else
        k_expand<M, C64, false><<<g_exp, kExpandThreads, 0, c->stream>>>(c->P);
    if (ev) cudaEventRecord(ev[3], c->stream);
    k_finalize<<<std::max(1, std::min(c->P.n_inst, 1024)), 256, 0, c->stream>>>(c->P, M * M, g_exp);
    if (ev) cudaEventRecord(ev[4], c->stream);
    return cudaGetLastError();
}

// History tables of one window length staged in the stream kernel's shared
// memory when they take at most kMaxStreamLut bytes (0: read from global).
size_t stream_lut_bytes(const qp_ctx *c, bool c64) {
    if (c->P.ndelta == 0) return 0;
    const size_t n = (size_t)c->P.nchunks * kLutEntries;
    const size_t b = c64 ? 2 * n * sizeof(float2) : (size_t)c->P.ndelta * n * sizeof(double2);
    return b <= kMaxStreamLut ? b : 0;
}

// Grid of the stream kernel: every block resident (tiles are taken by
// ticket, so blocks beyond the co-resident count would only start after a
// first wave), at most blocks_per_sm per SM and kMaxExpandBlocks in all.
template <int M, bool C64, int NX, int S>
cudaError_t launch_stream_kernel(qp_ctx *c, int blocks_per_sm) {
    using Lay = StreamLayout<M, C64, NX, S>;
    const void *fn = (const void *)k_stream_step<M, C64, NX, S>;
    const size_t lutb = stream_lut_bytes(c, C64);
    const size_t sm = Lay::bytes + lutb;
    if (c->scache_fn != fn || c->scache_smem != sm) {
        // the attribute is a property of the function: set it to the most
        // any context may ask for, so that contexts do not undo each other
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(Lay::bytes + kMaxStreamLut));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kStreamThreads, sm);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        c->scache_fn = fn;
        c->scache_smem = sm;
        c->scache_res = nb;
    }
    const int g = std::min(c->nsm * std::min(blocks_per_sm, c->scache_res), kMaxExpandBlocks);
    k_stream_step<M, C64, NX, S><<<g, kStreamThreads, sm, c->stream>>>(c->P, lutb ? 1 : 0);
    return cudaGetLastError();
}

// Batched stream kernel: an ordinary launch of one step (every block
// resident, at most blocks_per_sm per SM), or (coop) one cooperative launch
// of nsteps steps over at most persistent_blocks co-resident blocks.
// Dynamic shared memory: the tile buffers, then the per-instance sums and
// the regions' first tiles.
template <int M, bool C64, int S>
cudaError_t launch_stream_batch_kernel(qp_ctx *c, int nsteps, bool coop) {
    using Lay = StreamLayout<M, C64, 1, S>;
    constexpr int MM = M * M;
    const void *fn = (const void *)k_stream_batch<M, C64, S>;
    auto extra = [](int ni) { return Lay::a16((size_t)ni * (MM + 1) * 16) + ((size_t)ni * MM + 1) * 4; };
    const size_t sm = Lay::bytes + extra(c->P.n_inst);
    if (c->scache_fn != fn || c->scache_smem != sm) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(Lay::bytes + extra(kMaxInst)));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kStreamThreads, sm);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        c->scache_fn = fn;
        c->scache_smem = sm;
        c->scache_res = nb;
    }
    if (coop) {
        const int g = std::min(std::min(c->persist_grid, c->nsm * c->scache_res), kMaxExpandBlocks);
        Params P = c->P;
        void *args[] = {(void *)&P, (void *)&nsteps};
        return cudaLaunchCooperativeKernel(fn, dim3(g), dim3(kStreamThreads), args, sm, c->stream);
    }
    const int g = std::min(c->nsm * std::min(c->bps_exp, c->scache_res), kMaxExpandBlocks);
    k_stream_batch<M, C64, S><<<g, kStreamThreads, sm, c->stream>>>(c->P, 1);
    return cudaGetLastError();
}

template <int M, bool C64>
cudaError_t launch_stream_batch_t(qp_ctx *c, int nsteps, bool coop) {
    return c->stream_tile == 1024 ? launch_stream_batch_kernel<M, C64, 1024>(c, nsteps, coop)
                                  : launch_stream_batch_kernel<M, C64, 512>(c, nsteps, coop);
}

cudaError_t launch_stream_batch(qp_ctx *c, int nsteps, bool coop) {
    const bool c64 = c->cfg.precision == QP_C64;
    switch (c->cfg.M) {
        case 2: return c64 ? launch_stream_batch_t<2, true>(c, nsteps, coop) : launch_stream_batch_t<2, false>(c, nsteps, coop);
        case 3: return c64 ? launch_stream_batch_t<3, true>(c, nsteps, coop) : launch_stream_batch_t<3, false>(c, nsteps, coop);
        default: return c64 ? launch_stream_batch_t<4, true>(c, nsteps, coop) : launch_stream_batch_t<4, false>(c, nsteps, coop);
    }
}

template <int M, bool C64, int NX>
cudaError_t launch_stream_tile(qp_ctx *c) {
    switch (c->stream_tile) {
        case 256: return launch_stream_kernel<M, C64, NX, 256>(c, c->bps_exp);
        case 1024: return launch_stream_kernel<M, C64, NX, 1024>(c, c->bps_exp);
        default: return launch_stream_kernel<M, C64, NX, 512>(c, c->bps_exp);
    }
}

// The regular stream kernel (M = 2, no filter): every block resident, at
// most kMaxExpandBlocks (block partials).
template <bool C64>
cudaError_t launch_stream_regular(qp_ctx *c) {
    const void *fn = (const void *)k_stream_regular<2, C64>;
    const size_t lutb = stream_lut_bytes(c, C64);
    if (c->rcache_fn != fn || c->rcache_smem != lutb) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxStreamLut);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kRegThreads, lutb);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        c->rcache_fn = fn;
        c->rcache_smem = lutb;
        c->rcache_res = nb;
    }
    const int g = std::min(c->nsm * c->rcache_res, kMaxExpandBlocks);
    k_stream_regular<2, C64><<<g, kRegThreads, lutb, c->stream>>>(c->P, lutb ? 1 : 0);
    return cudaGetLastError();
}

// One step of the stream engine: the regular kernel where the configuration
// allows regular steps (events 0 -> 1), then the tile kernel (events 2 -> 3),
// which returns at once when the regular kernel took the step.
template <int M, typename Amp>
cudaError_t launch_stream_t(qp_ctx *c, cudaEvent_t *ev) {
    constexpr bool C64 = sizeof(Amp) == sizeof(float2);
    if (ev) cudaEventRecord(ev[0], c->stream);
    if constexpr (M == 2) {
        if (c->P.reg_fill) {
            cudaError_t e = launch_stream_regular<C64>(c);
            if (e != cudaSuccess) return e;
        }
    }
    if (ev) {
        cudaEventRecord(ev[1], c->stream);
        cudaEventRecord(ev[2], c->stream);
    }
    cudaError_t e;
    if (c->P.n_inst > 1) {
        e = launch_stream_batch_t<M, C64>(c, 1, false);
    } else if constexpr (M == 2) {
        e = c->stream_nx == 4 ? launch_stream_tile<M, C64, 4>(c) : launch_stream_tile<M, C64, 1>(c);
    } else {
        e = launch_stream_tile<M, C64, 1>(c);
    }
    if (e != cudaSuccess) return e;
    if (ev) {
        cudaEventRecord(ev[3], c->stream);
        cudaEventRecord(ev[4], c->stream);
    }
    return cudaGetLastError();
}

// One post-merging step (events: 0 extension, 1 sort, 2 reduce by key,
// 3 publish, 4 end).  The number of radix passes covers the widest key (the
// whole window, b dkmax bits); passes beyond the step's key bits return at
// once on the device.
template <int M, bool C64>
cudaError_t launch_post_t(qp_ctx *c, cudaEvent_t *ev) {
    const int g_exp = std::min(c->nsm * c->bps_exp, kMaxExpandBlocks);
    const int gs = (int)std::min<long long>(c->L.max_chunks, (long long)c->nsm * 4);
    const int gc = (int)std::min<long long>(((long long)256 * c->L.max_chunks + kScanSeg - 1) / kScanSeg,
                                            (long long)c->nsm * 2);
    const int gk = c->nsm * 4;
    const int npass = (c->P.b * c->cfg.dkmax + 7) / 8;
    if (ev) cudaEventRecord(ev[0], c->stream);
    k_post_expand<M, C64><<<g_exp, kExpandThreads, 0, c->stream>>>(c->P);
    if (ev) cudaEventRecord(ev[1], c->stream);
    k_post_keys<<<gk, 256, 0, c->stream>>>(c->P);
    for (int pass = 0; pass < npass; ++pass) {
        k_rs_hist<<<gs, kSortThreads, 0, c->stream>>>(c->P, pass);
        k_scan_part<<<gc, kScanThreads, 0, c->stream>>>(c->P, c->P.rs_hist, 0, pass);
        k_scan_top<<<1, kScanThreads, 0, c->stream>>>(c->P, 0, pass);
        k_scan_down<<<gc, kScanThreads, 0, c->stream>>>(c->P, c->P.rs_hist, 0, pass);
        k_rs_scatter<<<gs, kSortThreads, 0, c->stream>>>(c->P, pass);
    }
    if (ev) cudaEventRecord(ev[2], c->stream);
    k_rbk_heads<<<gs, kSortThreads, 0, c->stream>>>(c->P);
    k_scan_part<<<gc, kScanThreads, 0, c->stream>>>(c->P, c->P.rbk_heads, 1, 0);
    k_scan_top<<<1, kScanThreads, 0, c->stream>>>(c->P, 1, 0);
    k_scan_down<<<gc, kScanThreads, 0, c->stream>>>(c->P, c->P.rbk_heads, 1, 0);
    k_rbk_write<C64><<<gs, kSortThreads, 0, c->stream>>>(c->P);
    if (ev) cudaEventRecord(ev[3], c->stream);
    k_post_publish<<<1, 256, 0, c->stream>>>(c->P, M * M, g_exp);
    if (ev) cudaEventRecord(ev[4], c->stream);
    return cudaGetLastError();
}

cudaError_t launch_step(qp_ctx *c, cudaEvent_t *ev = nullptr) {
    const bool c64 = c->cfg.precision == QP_C64;
    if (c->P.post) {
        switch (c->cfg.M) {
            case 2: return c64 ? launch_post_t<2, true>(c, ev) : launch_post_t<2, false>(c, ev);
            case 3: return c64 ? launch_post_t<3, true>(c, ev) : launch_post_t<3, false>(c, ev);
            default: return c64 ? launch_post_t<4, true>(c, ev) : launch_post_t<4, false>(c, ev);
        }
    }
    if (c->use_stream) {
        switch (c->cfg.M) {
            case 2: return c64 ? launch_stream_t<2, float2>(c, ev) : launch_stream_t<2, double2>(c, ev);
            case 3: return c64 ? launch_stream_t<3, float2>(c, ev) : launch_stream_t<3, double2>(c, ev);
            default: return c64 ? launch_stream_t<4, float2>(c, ev) : launch_stream_t<4, double2>(c, ev);
        }
    }
    switch (c->cfg.M) {
        case 2: return c64 ? launch_step_t<2, float2>(c, ev) : launch_step_t<2, double2>(c, ev);
        case 3: return c64 ? launch_step_t<3, float2>(c, ev) : launch_step_t<3, double2>(c, ev);
        default: return c64 ? launch_step_t<4, float2>(c, ev) : launch_step_t<4, double2>(c, ev);
    }
}

template <int M, bool C64>
cudaError_t launch_persistent_t(qp_ctx *c, int nsteps) {
    void *args[] = {(void *)&c->P, (void *)&nsteps};
    if (c->P.n_inst > 1)
        return cudaLaunchCooperativeKernel((const void *)k_step_persistent<M, C64, true>, dim3(c->persist_grid),
                                           dim3(kPersistThreads), args, batch_smem(c), c->stream);
    return cudaLaunchCooperativeKernel((const void *)k_step_persistent<M, C64, false>, dim3(c->persist_grid),
                                       dim3(kPersistThreads), args, 0, c->stream);
}

cudaError_t launch_persistent(qp_ctx *c, int nsteps) {
    const bool c64 = c->cfg.precision == QP_C64;
    switch (c->cfg.M) {
        case 2: return c64 ? launch_persistent_t<2, true>(c, nsteps) : launch_persistent_t<2, false>(c, nsteps);
        case 3: return c64 ? launch_persistent_t<3, true>(c, nsteps) : launch_persistent_t<3, false>(c, nsteps);
        default: return c64 ? launch_persistent_t<4, true>(c, nsteps) : launch_persistent_t<4, false>(c, nsteps);
    }
}

// Blocks of the persistent kernel: all must be co-resident (cooperative
// launch), at most kMaxExpandBlocks (rho partial buffer).
template <int M, bool C64>
int persistent_grid_t(int nsm, bool batch, size_t smem) {
    int nb = 0;
    cudaError_t e = batch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_persistent<M, C64, true>,
                                                                          kPersistThreads, smem)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_persistent<M, C64, false>,
                                                                          kPersistThreads, 0);
    if (e != cudaSuccess) return 0;
    return std::min(std::max(0, nb) * nsm, kMaxExpandBlocks);
}

// Batched kernels keep per-instance rho accumulators in dynamic shared memory.
template <int M, bool C64>
void allow_batch_smem_t(size_t smem) {
    if (smem <= 48 * 1024) return;
    cudaFuncSetAttribute(k_expand<M, C64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_step_persistent<M, C64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void allow_batch_smem(int M, bool c64, size_t smem) {
    switch (M) {
        case 2: c64 ? allow_batch_smem_t<2, true>(smem) : allow_batch_smem_t<2, false>(smem); break;
        case 3: c64 ? allow_batch_smem_t<3, true>(smem) : allow_batch_smem_t<3, false>(smem); break;
        default: c64 ? allow_batch_smem_t<4, true>(smem) : allow_batch_smem_t<4, false>(smem); break;
    }
}

int persistent_grid(int M, bool c64, int nsm, bool batch, size_t smem) {
    switch (M) {
        case 2: return c64 ? persistent_grid_t<2, true>(nsm, batch, smem) : persistent_grid_t<2, false>(nsm, batch, smem);
        case 3: return c64 ? persistent_grid_t<3, true>(nsm, batch, smem) : persistent_grid_t<3, false>(nsm, batch, smem);
        default: return c64 ? persistent_grid_t<4, true>(nsm, batch, smem) : persistent_grid_t<4, false>(nsm, batch, smem);
    }
}

void set_mask_params(qp_ctx *c) {
    Params &P = c->P;
    const int b = P.b, dk = P.dkmax;
    std::vector<int> Pp;   // P' = {p-1 : p in P, p >= 1} plus 0; post-merging: P itself
    std::vector<char> in(dk, 0);
    in[0] = 1;
    for (int p : c->mask)
        if (P.post) in[p] = 1;
        else if (p >= 1) in[p - 1] = 1;
    unsigned long long pm = 0;
    for (int p = 0; p < dk; ++p)
        if (in[p]) {
            Pp.push_back(p);
            pm |= ((1ull << b) - 1ull) << (b * p);
        }
    P.pmask = pm | P.instmask;   // paths of different instances never merge
    // dense index: compress the runs of consecutive P' positions (then the
    // instance index)
    int nruns = 0, off = 0;
    bool ok = true;
    for (size_t i = 0; i < Pp.size();) {
        size_t j = i;
        while (j + 1 < Pp.size() && Pp[j + 1] == Pp[j] + 1) ++j;
        if (nruns == kMaxRuns) { ok = false; break; }
        const int len = int(j - i + 1);
        P.run_shift[nruns] = b * Pp[i];
        P.run_mask[nruns] = (b * len >= 64) ? ~0ull : ((1ull << (b * len)) - 1ull);
        P.run_off[nruns] = off;
        off += b * len;
        ++nruns;
        i = j + 1;
    }
    if (P.n_inst > 1) {
        if (nruns == kMaxRuns) ok = false;
        else {
            const int ib = inst_bits(P.n_inst);
            P.run_shift[nruns] = P.inst_shift;
            P.run_mask[nruns] = (1ull << ib) - 1ull;
            P.run_off[nruns] = off;
            off += ib;
            ++nruns;
        }
    }
    P.nruns = nruns;
    P.dense = (ok && off <= (int)P.tcap_log2) ? 1 : 0;
    // stream engine: P' = prefix {0 .. k-1} plus at most one extra position
    // (M = 2: four sub-groups per run)
    int k = 0;
    while (k < (int)Pp.size() && Pp[k] == k) ++k;
    const int nextra = (int)Pp.size() - k;
    P.prefmask = (b * k >= 64) ? ~0ull : ((1ull << (b * k)) - 1ull);
    P.x_shift = nextra == 1 ? b * Pp[k] : -1;
    // (batches: the prefix alone)
    if (P.n_inst == 1) c->stream_nx = (nextra == 0 || (nextra == 1 && c->cfg.M == 2)) ? (nextra ? 4 : 1) : 0;
    else c->stream_nx = nextra == 0 ? 1 : 0;
    // regular steps (see Params, single problems): no filter; the merge form
    // needs P' = all positions but the oldest and a complete key set that
    // fits the buffers
    P.reg_fill = (c->cfg.theta == 0.0 && P.n_inst == 1) ? 1 : 0;
    P.reg_merge = (P.reg_fill && c->cfg.dkmax >= 2 && nextra == 0 && k == c->cfg.dkmax - 1) ? 1 : 0;
    P.full_n = 0;
    if (2.0 * c->cfg.dkmax * std::log2((double)c->cfg.M) < 62.0) {
        unsigned long long f = 1;
        for (int i = 0; i < 2 * c->cfg.dkmax; ++i) f *= (unsigned long long)c->cfg.M;
        if (f <= (unsigned long long)P.region_cap * (unsigned long long)(c->cfg.M * c->cfg.M)) P.full_n = f;
    }
    if (P.full_n == 0) P.reg_merge = 0;
    if (P.post) {   // the sort engine: no stream layout, no regular steps
        c->stream_nx = 0;
        P.reg_fill = P.reg_merge = 0;
        // more runs of consecutive positions than the packing holds: sort on
        // the masked key itself (up to its highest bit)
        P.post_compress = ok ? 1 : 0;
        P.post_bits_full = ok ? b * (int)Pp.size() : 64 - __builtin_clzll(pm);
    }
}

}  // namespace

// ================================================================= C ABI

extern "C" {

int qp_version(void) { return 100; }

const char *qp_status_string(qp_status s) {
    switch (s) {
        case QP_OK: return "ok";
        case QP_ERR_ARG: return "invalid argument";
        case QP_ERR_OOM: return "out of memory";
        case QP_ERR_CUDA: return "CUDA error";
        case QP_ERR_CAPACITY: return "capacity exceeded";
        case QP_ERR_TIMEOUT: return "device wait timed out";
        case QP_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

qp_status qp_workspace_size(const qp_config *cfg, size_t *bytes) {
    if (!bytes) return QP_ERR_ARG;
    if (validate(cfg)) return QP_ERR_ARG;
    *bytes = make_layout(cfg).total;
    return QP_OK;
}

qp_status qp_create(const qp_config *cfg, void *d_workspace, size_t bytes, void *cuda_stream, qp_ctx **out) {
    if (!out) return QP_ERR_ARG;
    *out = nullptr;
    if (validate(cfg)) return QP_ERR_ARG;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return QP_ERR_ARG;
    const Layout L = make_layout(cfg);
    if (bytes < L.total) return QP_ERR_OOM;
    qp_ctx *c = new (std::nothrow) qp_ctx();
    if (!c) return QP_ERR_OOM;
    c->cfg = *cfg;
    c->cfg.max_groups = cfg->max_groups ? cfg->max_groups : cfg->max_paths;
    c->cfg.rho_history = cfg->rho_history ? cfg->rho_history : 4096;
    c->cfg.q = nullptr;
    c->cfg.hs_re = c->cfg.hs_im = nullptr;
    const int M = cfg->M;
    c->q.assign(cfg->q, cfg->q + M);
    c->hs.resize(M * M);
    for (int i = 0; i < M * M; ++i) c->hs[i] = qp::cplx(cfg->hs_re[i], cfg->hs_im ? cfg->hs_im[i] : 0.0);
    c->U = qp::short_time_propagator(M, c->hs, cfg->dt);
    c->L = L;
    c->ws = static_cast<char *>(d_workspace);
    c->ws_bytes = bytes;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->use_graph = c->stream != nullptr && !getenv("QP_NO_GRAPH");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return QP_ERR_CUDA;
    }
    {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
        const int NI = std::max(1, cfg->n_inst);
        const size_t smem = NI > 1 ? (size_t)NI * (M * M + 1) * sizeof(double2) : 0;
        if (NI > 1) allow_batch_smem(M, cfg->precision == QP_C64, smem);
        c->persist_max = coop ? persistent_grid(M, cfg->precision == QP_C64, c->nsm, NI > 1, smem) : 0;
        c->persist_grid = std::min(c->persist_max, 2 * c->nsm);
        if (const char *bps = getenv("QP_PERSIST_BLOCKS_PER_SM")) {   // launch-shape override (tuning)
            const int want = atoi(bps) * c->nsm;
            if (want > 0 && want <= c->persist_max) c->persist_grid = want;
        }
        // default: the CUDA graph of the four step kernels (faster than the
        // persistent kernel's grid barriers when one step is launched at a time)
        c->use_persistent = c->persist_grid > 0 && getenv("QP_PERSISTENT") != nullptr;
    }
    Params &P = c->P;
    P.M = M;
    P.bs = bits_per_state(M);
    P.b = 2 * P.bs;
    P.dkmax = cfg->dkmax;
    P.nchunks = L.nchunks;
    P.tcap_log2 = L.tcap_log2;
    P.tcap_mask = L.tcap - 1;
    P.theta2 = cfg->theta * cfg->theta;
    P.max_paths = cfg->max_paths;
    P.max_groups = c->cfg.max_groups;
    P.rho_hist = c->cfg.rho_history;
    for (int k = 0; k < 2; ++k) {
        P.keys[k] = reinterpret_cast<unsigned long long *>(c->ws + L.keys[k]);
        P.amps[k] = c->ws + L.amps[k];
    }
    P.slots = reinterpret_cast<Slot *>(c->ws + L.slots);
    P.repk = reinterpret_cast<unsigned long long *>(c->ws + L.repk);
    P.slot_of = reinterpret_cast<unsigned int *>(c->ws + L.slot_of);
    P.groups = reinterpret_cast<unsigned int *>(c->ws + L.groups);
    P.lut = reinterpret_cast<const double2 *>(c->ws + L.lut);
    P.lutf = reinterpret_cast<const float2 *>(c->ws + L.lutf);
    P.lutf_lo = reinterpret_cast<const float2 *>(c->ws + L.lutlo);
    P.wtab = reinterpret_cast<const double2 *>(c->ws + L.wtab);
    P.wtabf = reinterpret_cast<const float4 *>(c->ws + L.wtabf);
    P.etab = reinterpret_cast<const double2 *>(c->ws + L.etab);
    {
        std::vector<double> dv;
        signed char dsel[16];
        for (int k = 0; k < 16; ++k) dsel[k] = -1;
        P.ndelta = distinct_deltas(M, cfg->q, &dv, dsel);
        set_equispaced(P, M, cfg->q, dv.data(), P.ndelta);
        for (int k = 0; k < 16; ++k) P.dsel[k] = dsel[k];
        for (int k = 0; k < kMaxDelta; ++k) P.deltaf[k] = k < P.ndelta ? (float)dv[k] : 0.f;
        c->deltas = dv;
    }
    P.theta2f = (float)(cfg->theta * cfg->theta);
    P.tie_rel = cfg->precision == QP_C64 ? kTieRelC64 : kTieRelFP64;
    P.rho_ring = reinterpret_cast<double2 *>(c->ws + L.rho);
    P.rho_part = reinterpret_cast<double2 *>(c->ws + L.rho_part);
    P.spart = reinterpret_cast<float4 *>(c->ws + L.spart);
    P.scount = reinterpret_cast<long long *>(c->ws + L.scount);
    P.inst_kept = reinterpret_cast<long long *>(c->ws + L.inst_kept);
    P.fin_count = reinterpret_cast<unsigned int *>(c->ws + L.fin_count);
    P.n_inst = std::max(1, cfg->n_inst);
    P.inst_shift = P.b * cfg->dkmax;
    P.instmask = P.n_inst > 1 ? (((1ull << inst_bits(P.n_inst)) - 1ull) << P.inst_shift) : 0ull;
    P.lut_stride = L.nlut;
    P.region_cap = (cfg->max_paths / ((long long)P.n_inst * M * M)) & ~15ll;   // region bases 16-entry aligned
    P.reg_n = reinterpret_cast<unsigned long long *>(c->ws + L.reg_n);
    P.tile_state = reinterpret_cast<unsigned long long *>(c->ws + L.tile_state);
    P.max_tiles = L.max_tiles;
    P.etab_stride = L.nlut * (size_t)std::max(1, L.nd);
    P.stats_ring = reinterpret_cast<StepRec *>(c->ws + L.stats);
    P.st = reinterpret_cast<DevState *>(c->ws + L.state);
    P.post = cfg->scheme == QP_POSTMERGE ? 1 : 0;
    if (P.post) {
        P.ckeys = reinterpret_cast<unsigned long long *>(c->ws + L.ckeys);
        P.camps = c->ws + L.camps;
        for (int k = 0; k < 2; ++k) {
            P.skey[k] = reinterpret_cast<unsigned long long *>(c->ws + L.skey[k]);
            P.sidx[k] = reinterpret_cast<unsigned int *>(c->ws + L.sidx[k]);
        }
        P.rs_hist = reinterpret_cast<unsigned int *>(c->ws + L.rs_hist);
        P.rs_part = reinterpret_cast<unsigned int *>(c->ws + L.rs_part);
        P.rbk_heads = reinterpret_cast<unsigned int *>(c->ws + L.rbk_heads);
    }
    c->mask.clear();
    for (int p = 0; p < cfg->dkmax; ++p) c->mask.push_back(p);
    set_mask_params(c);
    // device constants: q, U; zeroed state
    std::vector<double2> Ud(M * M);
    for (int i = 0; i < M * M; ++i) Ud[i] = make_double2(c->U[i].real(), c->U[i].imag());
    e = cudaMemcpyAsync(c->ws + L.q, c->q.data(), M * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ws + L.uprop, Ud.data(), M * M * sizeof(double2), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !c->deltas.empty())
        e = cudaMemcpyAsync(c->ws + L.deltas, c->deltas.data(), c->deltas.size() * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.state, 0, sizeof(DevState), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.fin_count, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.tile_state, 0, (size_t)L.max_tiles * M * M * 8, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete c;
        return QP_ERR_CUDA;
    }
    *out = c;
    return QP_OK;
}

void qp_destroy(qp_ctx *ctx) {
    if (!ctx) return;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->graph1) cudaGraphExecDestroy(ctx->graph1);
    if (ctx->hpin) cudaFreeHost(ctx->hpin);
    delete ctx;
}

qp_status qp_eta_from_bath(const qp_bath *bath, double dt, int n, double *eta_re, double *eta_im) {
    if (!bath || !eta_re || !eta_im || n < 1 || n > 4096) return QP_ERR_ARG;
    std::vector<qp::cplx> eta;
    if (qp::eta_from_bath(*bath, dt, n, eta)) return QP_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        eta_re[i] = eta[i].real();
        eta_im[i] = eta[i].imag();
    }
    return QP_OK;
}

static qp_status set_eta_one(qp_ctx *c, int inst, const double *re, const double *im, const double2 *eta0 = nullptr) {
    const int dk = c->cfg.dkmax, M = c->cfg.M, MM = M * M;
    std::vector<double2> e(dk);
    for (int i = 0; i < dk; ++i) {
        if (!std::isfinite(re[i]) || !std::isfinite(im[i])) return fail(c, QP_ERR_ARG, "eta must be finite");
        e[i] = make_double2(re[i], im[i]);
    }
    const Params &P = c->P;
    double2 *ed = reinterpret_cast<double2 *>(c->ws + c->L.eta) + (size_t)inst * dk;
    QP_CUDA(c, cudaMemcpyAsync(ed, e.data(), dk * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    const double *qd = reinterpret_cast<const double *>(c->ws + c->L.q);
    double2 *lut = reinterpret_cast<double2 *>(c->ws + c->L.lut) + (size_t)inst * P.lut_stride;
    if (P.nchunks > 0) {
        k_build_lut<<<64, 256, 0, c->stream>>>(lut, reinterpret_cast<float2 *>(c->ws + c->L.lutf) + inst * P.lut_stride,
                                               reinterpret_cast<float2 *>(c->ws + c->L.lutlo) + inst * P.lut_stride, ed,
                                               qd, M, P.bs, P.b, dk, P.nchunks, eta0);
        QP_CUDA(c, cudaGetLastError());
    }
    k_build_w<<<1, 256, 0, c->stream>>>(reinterpret_cast<double2 *>(c->ws + c->L.wtab) + (size_t)inst * MM * MM,
                                        reinterpret_cast<float4 *>(c->ws + c->L.wtabf) + (size_t)inst * MM * MM,
                                        reinterpret_cast<const double2 *>(c->ws + c->L.uprop), ed, qd, M);
    QP_CUDA(c, cudaGetLastError());
    if (P.nchunks > 0 && P.ndelta > 0) {
        k_build_etab<<<256, 256, 0, c->stream>>>(reinterpret_cast<double2 *>(c->ws + c->L.etab) + inst * P.etab_stride,
                                                 lut, reinterpret_cast<const double *>(c->ws + c->L.deltas), P.ndelta,
                                                 dk, P.nchunks);
        QP_CUDA(c, cudaGetLastError());
    }
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    return QP_OK;
}

qp_status qp_set_eta(qp_ctx *c, const double *re, const double *im, int n) {
    if (!c) return QP_ERR_ARG;
    if (!re || !im || n < c->cfg.dkmax) return fail(c, QP_ERR_ARG, "need dkmax influence coefficients");
    c->sym = false;   // back to the right-box reading
    c->P.sym = 0;
    c->graph_dirty = true;
    for (int inst = 0; inst < c->P.n_inst; ++inst) {
        const qp_status st = set_eta_one(c, inst, re, im);
        if (st != QP_OK) return st;
    }
    c->have_eta = true;
    return QP_OK;
}

qp_status qp_Q_from_bath(const qp_bath *bath, double h, int n, double *re, double *im) {
    if (!bath || !re || !im || n < 1 || n > 8192) return QP_ERR_ARG;
    std::vector<qp::cplx> Q;
    if (qp::Q_from_bath(*bath, h, n, Q)) return QP_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        re[i] = Q[i].real();
        im[i] = Q[i].imag();
    }
    return QP_OK;
}

qp_status qp_set_end_points(qp_ctx *c, const double *qr, const double *qi, int n) {
    if (!c) return QP_ERR_ARG;
    const int dk = c->cfg.dkmax, M = c->cfg.M, MM = M * M;
    if (!qr || !qi || n < 2 * dk + 1) return fail(c, QP_ERR_ARG, "need Q at multiples of dt/2 up to 2 dkmax");
    if (c->P.n_inst > 1 || c->P.post || c->cfg.engine == QP_ENGINE_STREAM)
        return fail(c, QP_ERR_STATE, "the symmetric splitting runs on the merge-table engine, pre-merging order, "
                                     "single problems");
    std::vector<qp::cplx> Qh(n);
    for (int j = 0; j < n; ++j) {
        if (!std::isfinite(qr[j]) || !std::isfinite(qi[j])) return fail(c, QP_ERR_ARG, "Q must be finite");
        Qh[j] = qp::cplx(qr[j], qi[j]);
    }
    // interior (full-interval) coefficients, point 0 with an interior point,
    // the newest point with an interior point and with point 0 (memory cut at
    // lags >= dkmax); the corrections are end-point minus interior values
    std::vector<double> er(dk), ei(dk);
    std::vector<double2> eta0(dk), dE(dk), dE0(dk);
    std::vector<qp::cplx> eta(dk);
    eta[0] = Qh[2];
    for (int d = 1; d < dk; ++d) eta[d] = Qh[2 * d + 2] - 2.0 * Qh[2 * d] + Qh[2 * d - 2];
    for (int d = 0; d < dk; ++d) {
        er[d] = eta[d].real();
        ei[d] = eta[d].imag();
    }
    eta0[0] = dE[0] = dE0[0] = make_double2(0.0, 0.0);
    for (int k = 1; k < dk; ++k) {
        const qp::cplx e0 = Qh[2 * k + 1] - Qh[2 * k] - Qh[2 * k - 1] + Qh[2 * k - 2];
        const qp::cplx eE = Qh[2 * k + 1] - Qh[2 * k - 1] - Qh[2 * k] + Qh[2 * k - 2];
        const qp::cplx eE0 = Qh[2 * k] - 2.0 * Qh[2 * k - 1] + Qh[2 * k - 2];
        eta0[k] = make_double2(e0.real(), e0.imag());
        dE[k] = make_double2((eE - eta[k]).real(), (eE - eta[k]).imag());
        dE0[k] = make_double2((eE0 - e0).real(), (eE0 - e0).imag());
    }
    const qp::cplx dS = Qh[1] - eta[0];   // the newest point's half interval against a full one
    std::vector<double2> wE((size_t)MM * MM);
    std::vector<float4> wEf((size_t)MM * MM);
    for (int k = 0; k < MM; ++k) {
        const int a = k / M, b = k % M;
        const double qa = c->q[a], qb = c->q[b];
        const qp::cplx z = -(qa - qb) * (dS * qa - std::conj(dS) * qb);
        const qp::cplx f = std::exp(z);
        for (int par = 0; par < MM; ++par) {
            wE[(size_t)k * MM + par] = make_double2(f.real(), f.imag());
            const float hx = (float)f.real(), hy = (float)f.imag();
            wEf[(size_t)k * MM + par] = make_float4(hx, hy, (float)(f.real() - (double)hx), (float)(f.imag() - (double)hy));
        }
    }
    const Params &P = c->P;
    double2 *eta0d = reinterpret_cast<double2 *>(c->ws + c->L.eta0d);
    double2 *dEd = reinterpret_cast<double2 *>(c->ws + c->L.dEd);
    double2 *dE0d = reinterpret_cast<double2 *>(c->ws + c->L.dE0d);
    QP_CUDA(c, cudaMemcpyAsync(eta0d, eta0.data(), dk * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaMemcpyAsync(dEd, dE.data(), dk * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaMemcpyAsync(dE0d, dE0.data(), dk * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaMemcpyAsync(c->ws + c->L.wEt, wE.data(), wE.size() * sizeof(double2), cudaMemcpyHostToDevice,
                               c->stream));
    QP_CUDA(c, cudaMemcpyAsync(c->ws + c->L.wEtf, wEf.data(), wEf.size() * sizeof(float4), cudaMemcpyHostToDevice,
                               c->stream));
    // the propagation's own tables, with point 0 on its half interval
    qp_status st = set_eta_one(c, 0, er.data(), ei.data(), eta0d);
    if (st != QP_OK) return st;
    // the correction's history tables (and their exp(-delta T) products for FP64)
    const double *qd = reinterpret_cast<const double *>(c->ws + c->L.q);
    double2 *lutE = reinterpret_cast<double2 *>(c->ws + c->L.lutE);
    if (P.nchunks > 0) {
        k_build_lut<<<64, 256, 0, c->stream>>>(lutE, reinterpret_cast<float2 *>(c->ws + c->L.lutEf),
                                               reinterpret_cast<float2 *>(c->ws + c->L.lutElo), dEd, qd, M, P.bs, P.b,
                                               dk, P.nchunks, dE0d);
        QP_CUDA(c, cudaGetLastError());
        if (P.ndelta > 0) {
            k_build_etab<<<256, 256, 0, c->stream>>>(reinterpret_cast<double2 *>(c->ws + c->L.etabE), lutE,
                                                     reinterpret_cast<const double *>(c->ws + c->L.deltas), P.ndelta,
                                                     dk, P.nchunks);
            QP_CUDA(c, cudaGetLastError());
        }
    }
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->P.lutE = lutE;
    c->P.lutEf = reinterpret_cast<const float2 *>(c->ws + c->L.lutEf);
    c->P.lutElo = reinterpret_cast<const float2 *>(c->ws + c->L.lutElo);
    c->P.etabE = reinterpret_cast<const double2 *>(c->ws + c->L.etabE);
    c->P.wEt = reinterpret_cast<const double2 *>(c->ws + c->L.wEt);
    c->P.wEtf = reinterpret_cast<const float4 *>(c->ws + c->L.wEtf);
    c->P.sym = 1;
    c->sym = true;
    c->eta00 = Qh[1];
    c->have_eta = true;
    c->graph_dirty = true;
    return QP_OK;
}

qp_status qp_set_eta_instance(qp_ctx *c, int inst, const double *re, const double *im, int n) {
    if (!c) return QP_ERR_ARG;
    if (inst < 0 || inst >= c->P.n_inst) return fail(c, QP_ERR_ARG, "instance index out of range");
    if (!re || !im || n < c->cfg.dkmax) return fail(c, QP_ERR_ARG, "need dkmax influence coefficients");
    if (!c->have_eta) return fail(c, QP_ERR_STATE, "qp_set_eta (all instances) must come first");
    return set_eta_one(c, inst, re, im);
}

qp_status qp_set_mask(qp_ctx *c, const int *positions, int n) {
    if (!c) return QP_ERR_ARG;
    const int dk = c->cfg.dkmax;
    std::vector<int> m;
    if (!positions || n == 0) {
        for (int p = 0; p < dk; ++p) m.push_back(p);
    } else {
        if (n < 0 || n > dk) return fail(c, QP_ERR_ARG, "mask size out of range");
        std::vector<char> seen(dk, 0);
        for (int i = 0; i < n; ++i) {
            const int p = positions[i];
            if (p < 0 || p >= dk) return fail(c, QP_ERR_ARG, "mask position out of [0, dkmax)");
            seen[p] = 1;
        }
        if (!seen[0] || (dk >= 2 && !seen[1])) return fail(c, QP_ERR_ARG, "mask must contain positions 0 and 1");
        for (int p = 0; p < dk; ++p)
            if (seen[p]) m.push_back(p);
    }
    const std::vector<int> old = c->mask;
    c->mask = m;
    set_mask_params(c);
    if (c->have_state && c->use_stream && c->stream_nx == 0) {
        c->mask = old;
        set_mask_params(c);
        return fail(c, QP_ERR_STATE, "the running stream-engine propagation cannot take this mask (restart with "
                                     "qp_set_rho0 after choosing the merge-table engine)");
    }
    c->graph_dirty = true;
    return QP_OK;
}

qp_status qp_set_rho0(qp_ctx *c, const double *re, const double *im) {
    if (!c) return QP_ERR_ARG;
    if (!re) return fail(c, QP_ERR_ARG, "rho0 required");
    if (!c->have_eta) return fail(c, QP_ERR_STATE, "qp_set_eta must come before qp_set_rho0");
    const int M = c->cfg.M, MM = M * M, NI = c->P.n_inst;
    const int bs = c->P.bs;
    std::vector<unsigned long long> keys;
    std::vector<double2> amps, rho((size_t)NI * MM);
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
            const double x = re[a * M + b], y = im ? im[a * M + b] : 0.0;
            if (!std::isfinite(x) || !std::isfinite(y)) return fail(c, QP_ERR_ARG, "rho0 must be finite");
            for (int i = 0; i < NI; ++i) rho[(size_t)i * MM + a * M + b] = make_double2(x, y);
        }
    long long nnz = 0;
    for (int i = 0; i < NI; ++i)
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) {
                const double2 v = rho[(size_t)i * MM + a * M + b];
                if (v.x != 0.0 || v.y != 0.0) {
                    const unsigned long long ib = NI > 1 ? ((unsigned long long)i << c->P.inst_shift) : 0ull;
                    keys.push_back(ib | (unsigned long long)(a | (b << bs)));
                    amps.push_back(v);
                    if (i == 0) ++nnz;
                }
            }
    if ((int64_t)keys.size() > c->cfg.max_paths) return fail(c, QP_ERR_CAPACITY, "rho0 exceeds max_paths");
    // engine of this propagation
    if (!c->P.post && c->cfg.engine == QP_ENGINE_STREAM && c->stream_nx == 0)
        return fail(c, QP_ERR_ARG, "the stream engine needs a mask whose P' is a prefix {0..k-1} plus at most one "
                                   "extra position (M = 2; batches: the prefix alone)");
    c->use_stream = !c->P.post && !c->sym &&
                    (c->cfg.engine == QP_ENGINE_STREAM || (c->cfg.engine == QP_ENGINE_AUTO && c->stream_nx > 0));
    if (c->use_stream && c->P.region_cap < 1) return fail(c, QP_ERR_CAPACITY, "max_paths < 16 M*M (stream engine)");
    c->P.stream = c->use_stream ? 1 : 0;
    c->graph_dirty = true;
    const size_t n = keys.size();
    const size_t ab = c->cfg.precision == QP_C64 ? sizeof(float2) : sizeof(double2);
    if (c->sym) {   // point 0 on its half interval: its self factor in the stored amplitudes
        for (size_t i = 0; i < n; ++i) {
            const int a = (int)(keys[i] & ((1u << bs) - 1u)), b = (int)((keys[i] >> bs) & ((1u << bs) - 1u));
            const double qa = c->q[a], qb = c->q[b];
            const qp::cplx f = std::exp(-(qa - qb) * (c->eta00 * qa - std::conj(c->eta00) * qb)) *
                               qp::cplx(amps[i].x, amps[i].y);
            amps[i] = make_double2(f.real(), f.imag());
        }
    }
    std::vector<float2> af(n);
    for (size_t i = 0; i < n; ++i) af[i] = make_float2((float)amps[i].x, (float)amps[i].y);
    const void *asrc = c->cfg.precision == QP_C64 ? (const void *)af.data() : (const void *)amps.data();
    DevState s{};
    s.n_cur = n;
    if (c->use_stream) {   // one path per region (instance, newest point a*M + b); keys without the instance
        std::vector<unsigned long long> rn((size_t)2 * NI * MM, 0ull);
        for (size_t i = 0; i < n; ++i) {
            const int a = (int)(keys[i] & ((1u << bs) - 1u)), b = (int)((keys[i] >> bs) & ((1u << bs) - 1u));
            const int inst = NI > 1 ? (int)(keys[i] >> c->P.inst_shift) : 0;
            const size_t reg = (size_t)inst * MM + (size_t)(a * M + b);
            keys[i] &= ~c->P.instmask;
            QP_CUDA(c, cudaMemcpyAsync(c->P.keys[0] + reg * c->P.region_cap, &keys[i], 8, cudaMemcpyHostToDevice,
                                       c->stream));
            QP_CUDA(c, cudaMemcpyAsync(static_cast<char *>(c->P.amps[0]) + reg * c->P.region_cap * ab,
                                       static_cast<const char *>(asrc) + i * ab, ab, cudaMemcpyHostToDevice, c->stream));
            rn[reg] = 1;
        }
        QP_CUDA(c, cudaMemcpyAsync(c->P.reg_n, rn.data(), rn.size() * 8, cudaMemcpyHostToDevice, c->stream));
        QP_CUDA(c, cudaStreamSynchronize(c->stream));   // rn and keys are host temporaries
    } else {
        QP_CUDA(c, cudaMemcpyAsync(c->P.keys[0], keys.data(), n * 8, cudaMemcpyHostToDevice, c->stream));
        QP_CUDA(c, cudaMemcpyAsync(c->P.amps[0], asrc, n * ab, cudaMemcpyHostToDevice, c->stream));
    }
    QP_CUDA(c, cudaMemcpyAsync(c->P.st, &s, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaMemcpyAsync(c->P.rho_ring, rho.data(), (size_t)NI * MM * sizeof(double2), cudaMemcpyHostToDevice,
                               c->stream));
    std::vector<long long> kept0(NI, nnz);
    QP_CUDA(c, cudaMemcpyAsync(c->P.inst_kept, kept0.data(), NI * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaMemsetAsync(c->P.fin_count, 0, sizeof(unsigned int), c->stream));
    // look-back words are tagged with the step number, which restarts at 0:
    // words of an earlier propagation must not pass for this one's
    QP_CUDA(c, cudaMemsetAsync(c->P.tile_state, 0, (size_t)c->L.max_tiles * M * M * 8, c->stream));
    StepRec r0{0, 0, 0, (long long)n, (long long)n};
    QP_CUDA(c, cudaMemcpyAsync(c->P.stats_ring, &r0, sizeof(StepRec), cudaMemcpyHostToDevice, c->stream));
    k_clear_table<<<c->nsm * 4, 256, 0, c->stream>>>(c->P.slots, c->P.repk, c->L.tcap);
    QP_CUDA(c, cudaGetLastError());
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_state = true;
    c->failed = false;
    c->host_t = 0;
    c->err.clear();
    return QP_OK;
}

static qp_status capture_graph(qp_ctx *c, int steps, cudaGraphExec_t *out) {
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaGraph_t g;
    QP_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < steps && le == cudaSuccess; ++s) le = launch_step(c);
    cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
    if (le != cudaSuccess) return fail(c, QP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(le));
    if (ce != cudaSuccess) return fail(c, QP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    cudaError_t ie = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(c, QP_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(ie));
    return QP_OK;
}

qp_status qp_step(qp_ctx *c, int nsteps) {
    if (!c) return QP_ERR_ARG;
    if (nsteps < 0) return fail(c, QP_ERR_ARG, "nsteps < 0");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "qp_set_rho0 must come before qp_step");
    if (c->failed) return fail(c, QP_ERR_STATE, "context holds a device error; call qp_set_rho0");
    if (nsteps == 0) return QP_OK;
    c->host_t += nsteps;
    if (c->use_persistent && !c->use_stream && !c->P.post) {
        const cudaError_t e = launch_persistent(c, nsteps);
        if (e != cudaSuccess) return fail(c, QP_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
        return QP_OK;
    }
    if (c->use_persistent && c->use_stream && c->P.n_inst > 1) {   // batched stream engine: all steps, one launch
        const cudaError_t e = launch_stream_batch(c, nsteps, true);
        if (e != cudaSuccess) return fail(c, QP_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
        return QP_OK;
    }
    if (c->use_graph) {
        if (c->graph_dirty || !c->graph1 || (c->graph_steps > 1 && !c->graph)) {
            qp_status st = capture_graph(c, 1, &c->graph1);
            if (st != QP_OK) return st;
            if (c->graph_steps > 1) {
                st = capture_graph(c, c->graph_steps, &c->graph);
                if (st != QP_OK) return st;
            }
            c->graph_dirty = false;
        }
        int left = nsteps;
        if (c->graph_steps > 1)
            for (; left >= c->graph_steps; left -= c->graph_steps) QP_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
        for (; left > 0; --left) QP_CUDA(c, cudaGraphLaunch(c->graph1, c->stream));
    } else {
        for (int s = 0; s < nsteps; ++s) {
            cudaError_t e = launch_step(c);
            if (e != cudaSuccess) return fail(c, QP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
        }
    }
    return QP_OK;
}

static qp_status check_state(qp_ctx *c, const DevState *s) {
    if (s->err) {
        c->failed = true;
        std::string what;
        if (s->err & kErrPaths) what += " path buffer (max_paths)";
        if (s->err & kErrGroups) what += " merge groups (max_groups)";
        if (s->err & kErrProbe) what += " merge table probe limit";
        if (what.empty())   // only a bounded wait gave up: a grid barrier or a look-back
            return fail(c, QP_ERR_TIMEOUT, "a bounded device wait (grid barrier or tile look-back) timed out at step " +
                                               std::to_string(s->t + 1));
        return fail(c, QP_ERR_CAPACITY, "capacity exceeded at step " + std::to_string(s->t + 1) + ":" + what);
    }
    return QP_OK;
}

static qp_status read_state(qp_ctx *c, DevState *s) {
    QP_CUDA(c, cudaMemcpyAsync(s, c->P.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->host_t = (int64_t)s->t;
    return check_state(c, s);
}

qp_status qp_sync(qp_ctx *c) {
    if (!c) return QP_ERR_ARG;
    DevState s;
    return read_state(c, &s);
}

qp_status qp_current(qp_ctx *c, int64_t *t, int64_t *n) {
    if (!c) return QP_ERR_ARG;
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    DevState s;
    qp_status r = read_state(c, &s);
    if (t) *t = (int64_t)s.t;
    if (n) *n = (int64_t)s.n_cur;
    return r;
}

qp_status qp_read_rho(qp_ctx *c, int64_t t0, int count, double *re, double *im) {
    if (!c) return QP_ERR_ARG;
    if (!re || !im || count < 0) return fail(c, QP_ERR_ARG, "bad output");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    if (c->use_stream) {   // the last step's rho may still be in block partials
        if (c->cfg.precision == QP_C64) k_rho_finalize<true><<<1, 256, 0, c->stream>>>(c->P, c->cfg.M * c->cfg.M);
        else k_rho_finalize<false><<<1, 256, 0, c->stream>>>(c->P, c->cfg.M * c->cfg.M);
        QP_CUDA(c, cudaGetLastError());
    }
    // one round trip: the state and the rows of steps t0 .. t0 + count - 1
    // (ring slots t mod R, at most two contiguous pieces, always inside the
    // ring) are copied to pinned memory together; the range and the error
    // flags are then checked on the copied state
    const int64_t R = c->cfg.rho_history;
    if (t0 < 0 || count > R) return fail(c, QP_ERR_ARG, "step outside the kept rho history");
    const size_t per = (size_t)c->P.n_inst * c->cfg.M * c->cfg.M;
    const size_t soff = (sizeof(DevState) + 15) & ~(size_t)15;
    const size_t need = soff + (size_t)count * per * sizeof(double2);
    if (need > c->hpin_bytes) {
        if (c->hpin) cudaFreeHost(c->hpin);
        c->hpin = nullptr;
        c->hpin_bytes = 0;
        QP_CUDA(c, cudaMallocHost(&c->hpin, need));
        c->hpin_bytes = need;
    }
    DevState *hs = static_cast<DevState *>(c->hpin);
    double2 *rows = reinterpret_cast<double2 *>(static_cast<char *>(c->hpin) + soff);
    QP_CUDA(c, cudaMemcpyAsync(hs, c->P.st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    for (int64_t done = 0; done < count;) {
        const int64_t slot = (t0 + done) % R, n = std::min<int64_t>(count - done, R - slot);
        QP_CUDA(c, cudaMemcpyAsync(rows + (size_t)done * per, c->P.rho_ring + (size_t)slot * per, (size_t)n * per * sizeof(double2),
                                   cudaMemcpyDeviceToHost, c->stream));
        done += n;
    }
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->host_t = (int64_t)hs->t;
    qp_status r = check_state(c, hs);
    if (r != QP_OK) return r;
    const int64_t tc = (int64_t)hs->t;
    if (t0 + count - 1 > tc || t0 <= tc - R) return fail(c, QP_ERR_ARG, "step outside the kept rho history");
    for (size_t i = 0; i < (size_t)count * per; ++i) {
        re[i] = rows[i].x;
        im[i] = rows[i].y;
    }
    return QP_OK;
}

qp_status qp_read_rho_async(qp_ctx *c, int64_t t0, int count, double *dst) {
    if (!c) return QP_ERR_ARG;
    if (!dst || count < 0) return fail(c, QP_ERR_ARG, "bad output");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    if (c->failed) return fail(c, QP_ERR_STATE, "context holds a device error; call qp_set_rho0");
    const int64_t R = c->cfg.rho_history, tc = c->host_t;
    if (t0 < 0 || count > R || t0 + count - 1 > tc || t0 <= tc - R)
        return fail(c, QP_ERR_ARG, "step outside the kept rho history");
    const size_t per = (size_t)c->P.n_inst * c->cfg.M * c->cfg.M;
    // page-locked dst the device can address: one kernel finalises and writes
    // the rows there (no copy); other memory: finalise, then cudaMemcpyAsync
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, dst) == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer) {
        double2 *ddst = static_cast<double2 *>(attr.devicePointer);
        const int MM = c->cfg.M * c->cfg.M, fin = c->use_stream ? 1 : 0;
        if (c->cfg.precision == QP_C64) k_rho_read_to<true><<<1, 256, 0, c->stream>>>(c->P, MM, fin, ddst, t0, (long long)count * per);
        else k_rho_read_to<false><<<1, 256, 0, c->stream>>>(c->P, MM, fin, ddst, t0, (long long)count * per);
        QP_CUDA(c, cudaGetLastError());
        return QP_OK;
    }
    cudaGetLastError();   // a pointer the runtime does not know is not an error here
    if (c->use_stream) {   // the last step's rho may still be in block partials
        if (c->cfg.precision == QP_C64) k_rho_finalize<true><<<1, 256, 0, c->stream>>>(c->P, c->cfg.M * c->cfg.M);
        else k_rho_finalize<false><<<1, 256, 0, c->stream>>>(c->P, c->cfg.M * c->cfg.M);
        QP_CUDA(c, cudaGetLastError());
    }
    double2 *out = reinterpret_cast<double2 *>(dst);
    for (int64_t done = 0; done < count;) {   // ring slots t mod R: at most two pieces
        const int64_t slot = (t0 + done) % R, n = std::min<int64_t>(count - done, R - slot);
        QP_CUDA(c, cudaMemcpyAsync(out + (size_t)done * per, c->P.rho_ring + (size_t)slot * per, (size_t)n * per * sizeof(double2),
                                   cudaMemcpyDeviceToHost, c->stream));
        done += n;
    }
    return QP_OK;
}

qp_status qp_read_instance_counts(qp_ctx *c, int64_t t, int64_t *kept) {
    if (!c) return QP_ERR_ARG;
    if (!kept) return fail(c, QP_ERR_ARG, "bad output");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    if (c->use_stream) {   // the last step's counts may still be in block partials
        if (c->cfg.precision == QP_C64) k_rho_finalize<true><<<1, 256, 0, c->stream>>>(c->P, c->cfg.M * c->cfg.M);
        else k_rho_finalize<false><<<1, 256, 0, c->stream>>>(c->P, c->cfg.M * c->cfg.M);
        QP_CUDA(c, cudaGetLastError());
    }
    DevState s;
    qp_status r = read_state(c, &s);
    if (r != QP_OK) return r;
    const int64_t R = c->cfg.rho_history, tc = (int64_t)s.t;
    if (t < 0 || t > tc || t <= tc - R) return fail(c, QP_ERR_ARG, "step outside the kept history");
    std::vector<long long> buf(c->P.n_inst);
    QP_CUDA(c, cudaMemcpyAsync(buf.data(), c->P.inst_kept + (size_t)(t % R) * c->P.n_inst,
                               c->P.n_inst * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->P.n_inst; ++i) kept[i] = buf[i];
    return QP_OK;
}

qp_status qp_read_stats(qp_ctx *c, int64_t t0, int count, qp_step_stats *out) {
    if (!c) return QP_ERR_ARG;
    if (!out || count < 0) return fail(c, QP_ERR_ARG, "bad output");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    DevState s;
    qp_status r = read_state(c, &s);
    if (r != QP_OK) return r;
    const int64_t R = c->cfg.rho_history, tc = (int64_t)s.t;
    if (t0 < 0 || t0 + count - 1 > tc || t0 <= tc - R) return fail(c, QP_ERR_ARG, "step outside the kept history");
    for (int k = 0; k < count; ++k) {
        StepRec rec;
        QP_CUDA(c, cudaMemcpyAsync(&rec, c->P.stats_ring + (t0 + k) % R, sizeof(StepRec), cudaMemcpyDeviceToHost,
                                   c->stream));
        QP_CUDA(c, cudaStreamSynchronize(c->stream));
        out[k].t = rec.t;
        out[k].groups = rec.groups;
        out[k].extended = rec.extended;
        out[k].kept = rec.kept;
        out[k].intermediate = rec.inter;
    }
    return QP_OK;
}

qp_status qp_export_paths(qp_ctx *c, uint64_t *keys, double *amps, int64_t cap, int64_t *n) {
    if (!c) return QP_ERR_ARG;
    if (!n || cap < 0 || (cap > 0 && (!keys || !amps))) return fail(c, QP_ERR_ARG, "bad output");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    DevState s;
    qp_status r = read_state(c, &s);
    if (r != QP_OK) return r;
    *n = (int64_t)s.n_cur;
    if ((int64_t)s.n_cur > cap) return fail(c, QP_ERR_CAPACITY, "export buffer too small");
    const int buf = (int)(s.t & 1);
    const size_t cnt = s.n_cur;
    const int MM = c->cfg.M * c->cfg.M;
    // contiguous pieces: the flat array, or the M*M regions of the stream engine
    std::vector<std::pair<size_t, size_t>> pieces;   // (device offset, count)
    std::vector<int> piece_inst;                       // stream batches: the instance of each piece
    if (c->use_stream) {
        const int nreg = c->P.n_inst * MM;
        std::vector<unsigned long long> rn((size_t)nreg);
        QP_CUDA(c, cudaMemcpyAsync(rn.data(), c->P.reg_n + (size_t)buf * nreg, (size_t)nreg * 8, cudaMemcpyDeviceToHost,
                                   c->stream));
        QP_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int r = 0; r < nreg; ++r)
            if (rn[r]) {
                pieces.push_back({(size_t)r * c->P.region_cap, (size_t)rn[r]});
                piece_inst.push_back(r / MM);
            }
    } else if (cnt) {
        pieces.push_back({0, cnt});
    }
    size_t o = 0;
    std::vector<float2> tmp(c->cfg.precision == QP_C64 ? cnt : 0);
    for (const auto &pc : pieces) {
        QP_CUDA(c, cudaMemcpyAsync(keys + o, c->P.keys[buf] + pc.first, pc.second * 8, cudaMemcpyDeviceToHost,
                                   c->stream));
        if (c->cfg.precision == QP_C64)
            QP_CUDA(c, cudaMemcpyAsync(tmp.data() + o, static_cast<float2 *>(c->P.amps[buf]) + pc.first,
                                       pc.second * sizeof(float2), cudaMemcpyDeviceToHost, c->stream));
        else
            QP_CUDA(c, cudaMemcpyAsync(amps + 2 * o, static_cast<double2 *>(c->P.amps[buf]) + pc.first,
                                       pc.second * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
        o += pc.second;
    }
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    if (o != cnt) return fail(c, QP_ERR_STATE, "region counts do not add up to the stored count");
    if (c->P.n_inst > 1 && c->use_stream) {   // the instance index above the path bits, as the merge-table engine keeps it
        size_t e = 0;
        for (size_t i = 0; i < pieces.size(); ++i)
            for (size_t j = 0; j < pieces[i].second; ++j, ++e)
                keys[e] |= (unsigned long long)piece_inst[i] << c->P.inst_shift;
    }
    for (size_t i = 0; i < tmp.size(); ++i) {
        amps[2 * i] = tmp[i].x;
        amps[2 * i + 1] = tmp[i].y;
    }
    return QP_OK;
}

// Holds the stream for about ns nanoseconds (one thread; at most 2^20
// sleeps of 64 ns), so that the host has enqueued a profiled step's events
// and kernels before the GPU reaches them and event intervals hold device
// time only.
__global__ void k_delay(unsigned long long ns) {
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < (1 << 20); ++i) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= ns) break;
        __nanosleep(64);
    }
}

qp_status qp_profile_steps(qp_ctx *c, int nsteps, double *kernel_ms, int nk) {
    if (!c) return QP_ERR_ARG;
    if (nsteps < 0 || !kernel_ms || nk < 0) return fail(c, QP_ERR_ARG, "bad arguments");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "qp_set_rho0 must come before qp_profile_steps");
    if (c->failed) return fail(c, QP_ERR_STATE, "context holds a device error; call qp_set_rho0");
    cudaEvent_t ev[kStepKernels + 1];
    for (int k = 0; k <= kStepKernels; ++k) QP_CUDA(c, cudaEventCreate(&ev[k]));
    qp_status st = QP_OK;
    for (int s = 0; s < nsteps && st == QP_OK; ++s) {
        k_delay<<<1, 1, 0, c->stream>>>(50000ull);
        cudaError_t e = launch_step(c, ev);
        ++c->host_t;
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[kStepKernels]);
        if (e != cudaSuccess) {
            st = fail(c, QP_ERR_CUDA, std::string("profile: ") + cudaGetErrorString(e));
            break;
        }
        for (int k = 0; k < kStepKernels && k < nk; ++k) {
            // stream engine: intervals without a kernel (1, 3, and 0 where
            // no regular map is launched) hold only event overhead
            if (c->use_stream && (k == 1 || k == 3 || (k == 0 && !(c->cfg.M == 2 && c->P.reg_fill)))) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            kernel_ms[k] += ms;
        }
    }
    for (int k = 0; k <= kStepKernels; ++k) cudaEventDestroy(ev[k]);
    if (st != QP_OK) return st;
    DevState ds;
    return read_state(c, &ds);
}

qp_status qp_get_tuning(qp_ctx *c, qp_tuning *out) {
    if (!c || !out) return QP_ERR_ARG;
    out->mode = c->use_persistent ? QP_LAUNCH_PERSISTENT : QP_LAUNCH_GRAPH;
    out->insert_blocks_per_sm = c->bps_ins;
    out->expand_blocks_per_sm = c->bps_exp;
    out->persistent_blocks = c->persist_grid;
    out->graph_steps = c->graph_steps;
    out->table_log2 = (int)c->P.tcap_log2;
    out->engine = c->use_stream ? QP_ENGINE_STREAM : QP_ENGINE_HASH;
    out->stream_tile = c->stream_tile;
    return QP_OK;
}

qp_status qp_set_tuning(qp_ctx *c, const qp_tuning *t) {
    if (!c || !t) return QP_ERR_ARG;
    if (t->mode != QP_LAUNCH_GRAPH && t->mode != QP_LAUNCH_PERSISTENT) return fail(c, QP_ERR_ARG, "unknown mode");
    if (t->mode == QP_LAUNCH_PERSISTENT && c->persist_max <= 0)
        return fail(c, QP_ERR_ARG, "cooperative launch not available on this device");
    if (t->mode == QP_LAUNCH_PERSISTENT && c->P.post)
        return fail(c, QP_ERR_ARG, "the post-merging scheme runs as CUDA graphs only");
    if (t->insert_blocks_per_sm < 1 || t->insert_blocks_per_sm > 32 || t->expand_blocks_per_sm < 1 ||
        c->nsm * t->expand_blocks_per_sm > kMaxExpandBlocks)
        return fail(c, QP_ERR_ARG, "blocks per SM out of range");
    if (t->mode == QP_LAUNCH_PERSISTENT && (t->persistent_blocks < 1 || t->persistent_blocks > c->persist_max))
        return fail(c, QP_ERR_ARG, "persistent blocks out of range (co-residency limit)");
    if (t->graph_steps < 1 || t->graph_steps > 1024) return fail(c, QP_ERR_ARG, "graph_steps out of range");
    if (t->table_log2 < 4 || t->table_log2 > (int)c->L.tcap_log2)
        return fail(c, QP_ERR_ARG, "table_log2 out of range (at most the workspace's table)");
    if (t->stream_tile != 0 && t->stream_tile != 256 && t->stream_tile != 512 && t->stream_tile != 1024)
        return fail(c, QP_ERR_ARG, "stream_tile must be 0 (unchanged), 256, 512 or 1024");
    if (t->stream_tile) c->stream_tile = t->stream_tile;
    c->use_persistent = t->mode == QP_LAUNCH_PERSISTENT;
    c->bps_ins = t->insert_blocks_per_sm;
    c->bps_exp = t->expand_blocks_per_sm;
    if (c->use_persistent) c->persist_grid = t->persistent_blocks;
    c->graph_steps = t->graph_steps;
    c->P.tcap_log2 = (unsigned)t->table_log2;
    c->P.tcap_mask = (1ull << t->table_log2) - 1ull;
    set_mask_params(c);   // the direct-index decision depends on the table size
    c->graph_dirty = true;
    return QP_OK;
}

namespace {
std::mutex g_tune_mutex;
std::map<std::string, qp_tuning> g_tune_cache;   // problem bucket -> best tuning

std::string tune_key(qp_ctx *c, long long n_paths) {
    int lg = 0;
    while ((1ll << lg) < std::max(1ll, n_paths)) ++lg;
    char buf[256];
    snprintf(buf, sizeof(buf), "M%d dk%d ni%d p%d th%d pm%llx n2^%d sm%d", c->cfg.M, c->cfg.dkmax, c->P.n_inst,
             c->cfg.precision, c->cfg.theta > 0.0 ? 1 : 0, c->P.pmask, lg, c->nsm);
    return buf;
}
}  // namespace

qp_status qp_autotune(qp_ctx *c, int trial_steps, int use_cache, qp_tuning *best, double *best_ms_per_step) {
    if (!c) return QP_ERR_ARG;
    if (trial_steps < 1 || trial_steps > 10000) return fail(c, QP_ERR_ARG, "trial_steps out of range");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "qp_set_rho0 must come before qp_autotune");
    if (c->failed) return fail(c, QP_ERR_STATE, "context holds a device error; call qp_set_rho0");
    int64_t t0 = 0, n0 = 0;
    qp_status st = qp_current(c, &t0, &n0);
    if (st != QP_OK) return st;
    const std::string key = tune_key(c, n0);
    if (use_cache) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            st = qp_set_tuning(c, &it->second);
            if (st == QP_OK) {
                if (best) *best = it->second;
                if (best_ms_per_step) *best_ms_per_step = -1.0;   // taken from the cache, not measured now
            }
            return st;
        }
    }
    // candidates: the step-kernel graph with several launch shapes and table
    // sizes, and the persistent kernel with several grid sizes
    std::vector<qp_tuning> cand;
    const int tl = (int)c->L.tcap_log2;
    std::vector<int> tables{tl};
    if (!c->P.dense)   // hashed tables: smaller tables trade probes for locality
        for (int d = 1; d <= 2; ++d) {
            long long need = 2;
            while (need < 2 * std::max<long long>(n0, 1)) need <<= 1;
            if ((1ll << (tl - d)) >= need) tables.push_back(tl - d);
        }
    const int gs = 8;
    if (c->P.post) {   // the sort engine: blocks per SM of the extension
        for (int be : {2, 4, 8})
            if (c->nsm * be <= kMaxExpandBlocks) cand.push_back(qp_tuning{QP_LAUNCH_GRAPH, c->bps_ins, be, c->persist_grid, gs, tl, 0, 0});
    } else if (c->use_stream && c->P.n_inst > 1) {   // batches: tile size; graphs of steps or one persistent launch
        for (int tile : {512, 1024}) {
            for (int be : {1, 2, 4})
                if (c->nsm * be <= kMaxExpandBlocks)
                    cand.push_back(qp_tuning{QP_LAUNCH_GRAPH, c->bps_ins, be, c->persist_grid, gs, tl, 0, tile});
            if (c->persist_max > 0)
                for (int pb : {1, 2})
                    cand.push_back(qp_tuning{QP_LAUNCH_PERSISTENT, c->bps_ins, c->bps_exp,
                                             std::min(c->persist_max, pb * c->nsm), gs, tl, 0, tile});
        }
    } else if (c->use_stream) {   // one kernel per step: tile size and blocks per SM
        for (int tile : {256, 512, 1024})
            for (int be : {1, 2, 4, 8}) {
                if (c->nsm * be > kMaxExpandBlocks) continue;
                cand.push_back(qp_tuning{QP_LAUNCH_GRAPH, c->bps_ins, be, c->persist_grid, gs, tl, 0, tile});
            }
    } else {
        for (int tb : tables)
            for (int bi : {2, 4, 8})
                for (int be : {2, 4, 8}) {
                    if (c->nsm * be > kMaxExpandBlocks) continue;
                    cand.push_back(qp_tuning{QP_LAUNCH_GRAPH, bi, be, c->persist_grid, gs, tb, 0, 0});
                }
        if (c->persist_max > 0)
            for (int pb : {1, 2, 4}) {
                const int blocks = std::min(c->persist_max, pb * c->nsm);
                cand.push_back(qp_tuning{QP_LAUNCH_PERSISTENT, 4, 4, blocks, gs, tl, 0, 0});
            }
    }
    qp_tuning save;
    qp_get_tuning(c, &save);
    cudaEvent_t e0, e1;
    QP_CUDA(c, cudaEventCreate(&e0));
    QP_CUDA(c, cudaEventCreate(&e1));
    double best_ms = 1e300;
    qp_tuning bt = save;
    for (const qp_tuning &cd : cand) {
        if (qp_set_tuning(c, &cd) != QP_OK) continue;
        if ((st = qp_step(c, 1)) != QP_OK) break;   // warm-up (captures the graphs)
        cudaEventRecord(e0, c->stream);
        if ((st = qp_step(c, trial_steps)) != QP_OK) break;
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(c, QP_ERR_CUDA, "autotune sync"); break; }
        DevState ds;
        if ((st = read_state(c, &ds)) != QP_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / trial_steps < best_ms) {
            best_ms = ms / trial_steps;
            bt = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != QP_OK) {
        qp_set_tuning(c, &save);
        return st;
    }
    st = qp_set_tuning(c, &bt);
    if (st != QP_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = bt;
    }
    if (best) *best = bt;
    if (best_ms_per_step) *best_ms_per_step = best_ms;
    return QP_OK;
}

qp_status qp_test_stall_barrier(qp_ctx *c) {
    if (!c) return QP_ERR_ARG;
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    // an arrival count that the last block can never complete: the next
    // persistent launch waits at its first grid barrier until the bounded
    // wait gives up
    const unsigned int poison = 0x40000000u;
    QP_CUDA(c, cudaMemcpyAsync(&c->P.st->bar_count, &poison, sizeof(poison), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    return QP_OK;
}

qp_status qp_test_stall_lookback(qp_ctx *c) {
    if (!c) return QP_ERR_ARG;
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    if (!c->use_stream) return fail(c, QP_ERR_STATE, "the propagation does not run on the stream engine");
    // the first tile of the next step publishes no look-back word: the
    // step's other tiles wait for it until their bounded wait gives up
    const unsigned int first = 1u;
    QP_CUDA(c, cudaMemcpyAsync(&c->P.st->stall_tile, &first, sizeof(first), cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    return QP_OK;
}

qp_status qp_partition_paths(qp_ctx *c, int n_ranks, uint64_t *d_keys, void *d_amps, int64_t cap, int64_t *counts) {
    if (!c) return QP_ERR_ARG;
    if (n_ranks < 1 || n_ranks > kMaxRanks || !counts || cap < 0 || (cap > 0 && (!d_keys || !d_amps)))
        return fail(c, QP_ERR_ARG, "bad arguments");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    if (c->use_stream || c->P.post || c->P.n_inst > 1)
        return fail(c, QP_ERR_STATE, "ranks need the merge-table engine, the pre-merging order and a single problem");
    DevState s;
    qp_status r = read_state(c, &s);
    if (r != QP_OK) return r;
    if ((int64_t)s.n_cur > cap) return fail(c, QP_ERR_CAPACITY, "partition buffer too small");
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c->ws + c->L.ranks);
    unsigned long long *base = cnt + kMaxRanks, *cursor = cnt + 2 * kMaxRanks;
    QP_CUDA(c, cudaMemsetAsync(cnt, 0, (size_t)n_ranks * 8, c->stream));
    const int g = std::max(1, std::min(c->nsm * 4, (int)((s.n_cur + 255) / 256)));
    k_part_count<<<g, 256, 0, c->stream>>>(c->P, (unsigned)n_ranks, cnt);
    QP_CUDA(c, cudaGetLastError());
    std::vector<unsigned long long> hc(n_ranks), hb(n_ranks);
    QP_CUDA(c, cudaMemcpyAsync(hc.data(), cnt, (size_t)n_ranks * 8, cudaMemcpyDeviceToHost, c->stream));
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    unsigned long long a = 0;
    for (int i = 0; i < n_ranks; ++i) {
        hb[i] = a;
        a += hc[i];
        counts[i] = (int64_t)hc[i];
    }
    QP_CUDA(c, cudaMemcpyAsync(base, hb.data(), (size_t)n_ranks * 8, cudaMemcpyHostToDevice, c->stream));
    QP_CUDA(c, cudaMemsetAsync(cursor, 0, (size_t)n_ranks * 8, c->stream));
    if (c->cfg.precision == QP_C64)
        k_part_scatter<float2><<<g, 256, 0, c->stream>>>(c->P, (unsigned)n_ranks, base, cursor,
                                                         reinterpret_cast<unsigned long long *>(d_keys), static_cast<float2 *>(d_amps));
    else
        k_part_scatter<double2><<<g, 256, 0, c->stream>>>(c->P, (unsigned)n_ranks, base, cursor,
                                                          reinterpret_cast<unsigned long long *>(d_keys), static_cast<double2 *>(d_amps));
    QP_CUDA(c, cudaGetLastError());
    QP_CUDA(c, cudaStreamSynchronize(c->stream));   // hb must outlive the copy; the caller reads the buffers next
    return QP_OK;
}

qp_status qp_import_paths(qp_ctx *c, const uint64_t *d_keys, const void *d_amps, int64_t n) {
    if (!c) return QP_ERR_ARG;
    if (n < 0 || (n > 0 && (!d_keys || !d_amps))) return fail(c, QP_ERR_ARG, "bad arguments");
    if (!c->have_state) return fail(c, QP_ERR_STATE, "no state");
    if (c->failed) return fail(c, QP_ERR_STATE, "context holds a device error; call qp_set_rho0");
    if (c->use_stream || c->P.post || c->P.n_inst > 1)
        return fail(c, QP_ERR_STATE, "ranks need the merge-table engine, the pre-merging order and a single problem");
    if (n > c->cfg.max_paths) return fail(c, QP_ERR_CAPACITY, "more paths than max_paths");
    DevState s;
    qp_status r = read_state(c, &s);
    if (r != QP_OK) return r;
    const int buf = (int)(s.t & 1);
    const size_t ab = c->cfg.precision == QP_C64 ? sizeof(float2) : sizeof(double2);
    if (n > 0) {
        QP_CUDA(c, cudaMemcpyAsync(c->P.keys[buf], d_keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
        QP_CUDA(c, cudaMemcpyAsync(c->P.amps[buf], d_amps, (size_t)n * ab, cudaMemcpyDeviceToDevice, c->stream));
    }
    k_set_count<<<1, 1, 0, c->stream>>>(c->P.st, (unsigned long long)n);
    QP_CUDA(c, cudaGetLastError());
    QP_CUDA(c, cudaStreamSynchronize(c->stream));
    return QP_OK;
}

const char *qp_last_error(const qp_ctx *c) { return c ? c->err.c_str() : "null context"; }

qp_status qp_test_widen(const float *in, double *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!in || !out)) || n > (int64_t)1 << 31) return QP_ERR_ARG;
    if (n == 0) return QP_OK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
    k_widen<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, out, n);
    return cudaGetLastError() == cudaSuccess ? QP_OK : QP_ERR_CUDA;
}


}  // extern "C"

// ================================================================= step without allocation
//
// qp_step_noalloc runs the same four step kernels as qp_step for one step,
// but on caller-provided input/output path buffers and with all scratch in
// one fixed-size array of device memory defined in this file, so that it
// neither allocates nor needs a workspace.  The paper has no counterpart; it
// exists for callers that cannot allocate device memory.

namespace {

constexpr long long kNaMaxPaths = 1ll << 20;   // stored paths of the input set
constexpr long long kNaMaxGroups = 1ll << 16;  // merge groups in one step
constexpr unsigned kNaTcapLog2 = 17;           // merge-table slots = 2^17
constexpr int kNaMaxDk = 16;                   // memory length
constexpr size_t kNaBytes = 20ull << 20;       // size of the fixed scratch (20 MiB)

// The fixed scratch.  In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

std::mutex g_na_mutex;
void *g_na_addr[256] = {};   // device address of g_na_scratch per device

qp_status na_scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (dev < 0 || dev >= 256) return QP_ERR_ARG;
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return QP_ERR_CUDA;
        g_na_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_addr[dev]);
    return QP_OK;
}

struct NaSetup {            // small set-up inputs, passed by value
    double2 eta[kNaMaxDk];
    double2 U[16];
    double q[4];
    double deltas[kMaxDelta];
    int dkmax, M, ndelta;
    unsigned long long t, n_in;
};

__global__ void k_na_setup(NaSetup s, double2 *eta, double *q, double2 *U, double *deltas, DevState *st,
                           unsigned int *fin_count) {
    const int i = threadIdx.x;
    if (i == 0) *fin_count = 0;
    if (i < s.dkmax) eta[i] = s.eta[i];
    if (i < s.M) q[i] = s.q[i];
    if (i < s.M * s.M) U[i] = s.U[i];
    if (i < s.ndelta) deltas[i] = s.deltas[i];
    if (i == 0) {
        DevState z{};
        z.t = s.t;
        z.n_cur = s.n_in;
        *st = z;
    }
}

}  // namespace

extern "C" qp_status qp_step_noalloc(const qp_config *cfg, const double *eta_re, const double *eta_im, int n_eta,
                                     const int *mask, int n_mask, int64_t t, const uint64_t *d_keys_in,
                                     const double *d_amps_in, int64_t n_in, uint64_t *d_keys_out, double *d_amps_out,
                                     int64_t cap_out, int64_t *n_out, double *rho_re, double *rho_im,
                                     void *cuda_stream) {
    if (validate(cfg) || cfg->precision != QP_FP64) return QP_ERR_ARG;
    const int M = cfg->M, dk = cfg->dkmax;
    if (dk > kNaMaxDk || !eta_re || !eta_im || n_eta < dk || !n_out || !rho_re || !rho_im) return QP_ERR_ARG;
    if (t < 0 || n_in < 0 || cap_out < 0) return QP_ERR_ARG;
    if (n_in > kNaMaxPaths) return QP_ERR_ARG;   // beyond the fixed scratch
    if ((n_in > 0 && (!d_keys_in || !d_amps_in)) || (cap_out > 0 && (!d_keys_out || !d_amps_out))) return QP_ERR_ARG;
    if ((const void *)d_keys_in == (const void *)d_keys_out || (const void *)d_amps_in == (const void *)d_amps_out)
        return QP_ERR_ARG;
    // mask -> P' bits and the compressed-index runs (fixed arrays)
    bool inP[kNaMaxDk] = {};
    if (!mask || n_mask == 0) {
        for (int p = 0; p < dk; ++p) inP[p] = true;
    } else {
        if (n_mask < 0 || n_mask > dk) return QP_ERR_ARG;
        for (int i = 0; i < n_mask; ++i) {
            if (mask[i] < 0 || mask[i] >= dk) return QP_ERR_ARG;
            inP[mask[i]] = true;
        }
        if (!inP[0] || (dk >= 2 && !inP[1])) return QP_ERR_ARG;
    }
    for (int i = 0; i < dk; ++i)
        if (!std::isfinite(eta_re[i]) || !std::isfinite(eta_im[i])) return QP_ERR_ARG;

    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QP_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QP_ERR_CUDA;
    unsigned char *base = nullptr;
    const qp_status ss = na_scratch_address(dev, &base);
    if (ss != QP_OK) return ss;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    Params P{};
    P.M = M;
    P.bs = bits_per_state(M);
    P.b = 2 * P.bs;
    P.dkmax = dk;
    P.nchunks = (dk - 1) * P.b > 0 ? ((dk - 1) * P.b + 7) / 8 : 0;
    P.tcap_log2 = kNaTcapLog2;
    P.tcap_mask = (1ull << kNaTcapLog2) - 1ull;
    P.theta2 = cfg->theta * cfg->theta;
    P.theta2f = (float)P.theta2;
    P.tie_rel = kTieRelFP64;
    P.max_paths = cap_out;
    P.max_groups = kNaMaxGroups;
    P.rho_hist = 2;
    P.n_inst = 1;
    P.inst_shift = P.b * dk;
    P.instmask = 0ull;
    {   // pre-merge positions P'' = {p-1 : p in P, p >= 1} plus 0, and dense runs
        bool inPp[kNaMaxDk] = {};
        inPp[0] = true;
        for (int p = 1; p < dk; ++p)
            if (inP[p]) inPp[p - 1] = true;
        unsigned long long pm = 0;
        int nruns = 0, off = 0;
        bool ok = true;
        for (int p = 0; p < dk;) {
            if (!inPp[p]) { ++p; continue; }
            int q2 = p;
            while (q2 + 1 < dk && inPp[q2 + 1]) ++q2;
            const int len = q2 - p + 1;
            for (int r = p; r <= q2; ++r) pm |= ((1ull << P.b) - 1ull) << (P.b * r);
            if (nruns == kMaxRuns) ok = false;
            else {
                P.run_shift[nruns] = P.b * p;
                P.run_mask[nruns] = (P.b * len >= 64) ? ~0ull : ((1ull << (P.b * len)) - 1ull);
                P.run_off[nruns] = off;
                ++nruns;
            }
            off += P.b * len;
            p = q2 + 1;
        }
        P.pmask = pm;
        P.nruns = nruns;
        P.dense = (ok && off <= (int)kNaTcapLog2) ? 1 : 0;
    }
    NaSetup su{};
    su.dkmax = dk;
    su.M = M;
    su.t = (unsigned long long)t;
    su.n_in = (unsigned long long)n_in;
    for (int i = 0; i < dk; ++i) su.eta[i] = make_double2(eta_re[i], eta_im[i]);
    for (int i = 0; i < M; ++i) su.q[i] = cfg->q[i];
    {
        qp::cplx H[16], U[16];
        for (int i = 0; i < M * M; ++i) H[i] = qp::cplx(cfg->hs_re[i], cfg->hs_im ? cfg->hs_im[i] : 0.0);
        qp::short_time_propagator(M, H, cfg->dt, U);   // fixed arrays: no allocation
        for (int i = 0; i < M * M; ++i) su.U[i] = make_double2(U[i].real(), U[i].imag());
        signed char dsel[16];
        for (int k = 0; k < 16; ++k) dsel[k] = -1;
        int nd = 0;
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) {
                const double d = cfg->q[a] - cfg->q[b];
                int idx = -1;
                if (d != 0.0) {
                    for (int k = 0; k < nd; ++k)
                        if (su.deltas[k] == d) idx = k;
                    if (idx < 0) { su.deltas[nd] = d; idx = nd++; }
                }
                dsel[a * M + b] = (signed char)idx;
            }
        su.ndelta = nd;
        P.ndelta = nd;
        set_equispaced(P, M, cfg->q, su.deltas, nd);
        for (int k = 0; k < 16; ++k) P.dsel[k] = dsel[k];
        for (int k = 0; k < kMaxDelta; ++k) P.deltaf[k] = k < nd ? (float)su.deltas[k] : 0.f;
    }
    // carve the fixed scratch (offsets from the limits above)
    const int MM = M * M;
    const size_t nlut = (size_t)kNaMaxDk * 8 * kLutEntries;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return base + o; };
    DevState *st = reinterpret_cast<DevState *>(take(sizeof(DevState)));
    P.slots = reinterpret_cast<Slot *>(take((1ull << kNaTcapLog2) * sizeof(Slot)));
    P.repk = reinterpret_cast<unsigned long long *>(take((1ull << kNaTcapLog2) * 8));
    P.slot_of = reinterpret_cast<unsigned int *>(take(kNaMaxPaths * 4));
    P.groups = reinterpret_cast<unsigned int *>(take(kNaMaxGroups * 4));
    double2 *lut = reinterpret_cast<double2 *>(take(nlut * sizeof(double2)));
    float2 *lutf = reinterpret_cast<float2 *>(take(nlut * sizeof(float2)));
    float2 *lutlo = reinterpret_cast<float2 *>(take(nlut * sizeof(float2)));
    double2 *etab = reinterpret_cast<double2 *>(take(nlut * kMaxDelta * sizeof(double2)));
    double2 *wtab = reinterpret_cast<double2 *>(take(256 * sizeof(double2)));
    float4 *wtabf = reinterpret_cast<float4 *>(take(256 * sizeof(float4)));
    double2 *Ud = reinterpret_cast<double2 *>(take(16 * sizeof(double2)));
    double2 *etad = reinterpret_cast<double2 *>(take(kNaMaxDk * sizeof(double2)));
    double *qd = reinterpret_cast<double *>(take(4 * sizeof(double)));
    double *deltad = reinterpret_cast<double *>(take(kMaxDelta * sizeof(double)));
    P.rho_ring = reinterpret_cast<double2 *>(take(2 * 16 * sizeof(double2)));
    // per-block partials of rho by step parity: M*M values and the survivor
    // count per block (the stride rho_part_of and phase_finalize use), for
    // the largest M
    P.rho_part = reinterpret_cast<double2 *>(take((size_t)2 * kMaxExpandBlocks * (16 + 1) * sizeof(double2)));
    P.stats_ring = reinterpret_cast<StepRec *>(take(2 * sizeof(StepRec)));
    P.inst_kept = reinterpret_cast<long long *>(take(2 * sizeof(long long)));
    P.fin_count = reinterpret_cast<unsigned int *>(take(sizeof(unsigned int)));
    if (off > kNaBytes) return QP_ERR_OOM;
    P.lut = lut;
    P.lutf = lutf;
    P.lutf_lo = lutlo;
    P.etab = etab;
    P.wtab = wtab;
    P.wtabf = wtabf;
    P.st = st;
    const int in = (int)(t & 1);
    P.keys[in] = const_cast<unsigned long long *>(reinterpret_cast<const unsigned long long *>(d_keys_in));
    P.amps[in] = const_cast<double *>(d_amps_in);
    P.keys[in ^ 1] = reinterpret_cast<unsigned long long *>(d_keys_out);
    P.amps[in ^ 1] = d_amps_out;

    // set-up (every call: the array keeps the previous call's contents)
    k_na_setup<<<1, 32, 0, stream>>>(su, etad, qd, Ud, deltad, st, P.fin_count);
    k_clear_table<<<nsm * 4, 256, 0, stream>>>(P.slots, P.repk, 1ull << kNaTcapLog2);
    if (P.nchunks > 0)
        k_build_lut<<<64, 256, 0, stream>>>(lut, lutf, lutlo, etad, qd, M, P.bs, P.b, dk, P.nchunks, nullptr);
    k_build_w<<<1, 256, 0, stream>>>(wtab, wtabf, Ud, etad, qd, M);
    if (P.nchunks > 0 && P.ndelta > 0) k_build_etab<<<256, 256, 0, stream>>>(etab, lut, deltad, P.ndelta, dk, P.nchunks);
    // the step: the same kernels as qp_step
    const int g_ins = nsm * 4;
    const int g_exp = std::min(nsm * 4, kMaxExpandBlocks);
    k_insert<double2><<<g_ins, kInsertThreads, 0, stream>>>(P);
    k_tiebreak<double2><<<g_ins, 256, 0, stream>>>(P);
    switch (M) {
        case 2: k_expand<2, false, false><<<g_exp, kExpandThreads, 0, stream>>>(P); break;
        case 3: k_expand<3, false, false><<<g_exp, kExpandThreads, 0, stream>>>(P); break;
        default: k_expand<4, false, false><<<g_exp, kExpandThreads, 0, stream>>>(P); break;
    }
    k_finalize<<<1, 256, 0, stream>>>(P, MM, g_exp);
    if (cudaGetLastError() != cudaSuccess) return QP_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return QP_ERR_CUDA;
    DevState s;
    double2 rho[16];
    if (cudaMemcpy(&s, st, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) return QP_ERR_CUDA;
    if (s.err) {
        *n_out = 0;
        return QP_ERR_CAPACITY;
    }
    if (cudaMemcpy(rho, P.rho_ring + ((t + 1) % 2) * MM, MM * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess)
        return QP_ERR_CUDA;
    *n_out = (int64_t)s.n_cur;
    for (int k = 0; k < MM; ++k) {
        rho_re[k] = rho[k].x;
        rho_im[k] = rho[k].y;
    }
    return QP_OK;
}
