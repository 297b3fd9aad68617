// rbl_internal.cuh -- device-side building blocks and the context layout of librbl.
//
// Everything here is written for sm_103a.  Decisions that select a neighbour (which
// side of a cutoff a pair falls on, which cell a particle is in, which batch is
// drawn) are made with explicitly rounded intrinsics (__fmul_rn, __fadd_rn,
// __int2float_rn) so that no compiler contraction can move a pair across a cutoff;
// the same rules are stated independently by the CPU oracle in the test-suite.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rbl.h"
#include "rbl_erfc_fit.cuh"

namespace rbl {

constexpr int kMaxP = 128;         // largest batch size
constexpr int kCellCap = 64;       // cells up to this size are sorted in local memory
constexpr int kBlock = 256;        // threads per block of the per-particle kernels
constexpr int kMinBlock = 64;      // smallest per-particle block: sizes the per-block partials
constexpr int kChunkGroups = 256;  // 64-thread groups per second-stage chunk of the per-replica sums
constexpr int kMaxStencil = 7;     // offsets per axis for K <= 3

constexpr int kTile = 256;         // particle slots per tile; every replica starts on a tile
constexpr int kTileShift = 8;
static_assert(kBlock == kTile, "a per-particle block covers exactly one tile");
constexpr int kMaxSeg = kMaxStencil * kMaxStencil;

// Device flags (bit positions in DevScalars::flags).
// kFlagNonFinite: a non-finite position, velocity or force, a binary32 force beyond
// the fixed-point range (|F| >= 2^29, overlapping particles), or a particle that left
// the box in one step (moved more than a box length).
enum : unsigned { kFlagOverflow = 1u, kFlagNonFinite = 2u, kFlagCellOverflow = 4u, kFlagRngLimit = 8u };
constexpr float kFixedRange = 536870880.0f; // below 2^29: |4 F| stays inside the int32 split of FixedAcc
constexpr float kEnergyRange = 274877906944.0f; // 2^38: |e 2^24| stays inside int64 with room for a sum

// Context-wide scalars living in device memory (one instance in the workspace).
struct DevScalars {
    unsigned flags;                 // kFlag* bits
    int rebuild;                    // 1 when some replica must rebuild before the next force
    unsigned long long step;        // step counter n (batch/noise counters), shared by all replicas
    unsigned obs_ticket;            // blocks of the observables launch done so far (zero between launches)
    unsigned pad_;
};

// Per-replica scalars living in device memory ([R] in the workspace).
struct RepScalars {
    unsigned long long fsum_q[3];   // FP32 path: sum of fixed-point forces (mod 2^64)
    unsigned long long ew_q[2];     // FP32 path: sums of the per-particle energy and virial
                                    // estimates in fixed point (scale 2^24, mod 2^64)
    double fcor[3];                 // mean force subtracted from every particle
    long long fcor_q[3];            // FP32 path: the net force Q (fixed point) as Q = N fcor_q + fcor_r,
    long long fcor_r[3];            // 0 <= fcor_r < N; tags < fcor_r subtract fcor_q + 1, the rest fcor_q
    double energy, virial;          // RBL estimates from the last evaluation
    double u_exact, w_exact;        // unsampled energy and virial (on demand)
    int rebuild;                    // 1 when this replica's lists must be rebuilt
    int nc_max, ns_max;             // longest rows at the last build (even past capacity)
    int m_max;                      // largest stencil population at the last build
    int t_max;                      // longest culled candidate table at the last build (shell sampling)
    unsigned long long ns_sum;      // total shell (or full) entries at the last build
    unsigned long long nc_sum;      // total core entries at the last build
    unsigned long long m_sum;       // sum over particles of their home cell's stencil population
    long long n_rebuild;            // builds so far
};

// One replica: an independent periodic system with its own box, temperature, seed
// and particle count (a context of one system is a batch of one).  Its particles
// occupy the slots [first, first + N) and the padding slots up to first + slots
// (slots = N rounded up to kTile), its cells the range [c0, c0 + ncell) followed by
// one pad cell that owns the padding slots, so that a single exclusive scan over
// every replica's cell counts places each replica at its own slots.
struct Box {
    double L[3], inv[3];            // inv = 2^32 / L
    float h[3];                     // L / 2^32 in binary32
    float c2f;                      // sqrt((1 - c1^2) T) in binary32
    unsigned long long seed;
    double T;
    int N, first, slots, in0;       // particles, first slot, slots, first row in packed caller arrays
    int c0, ncell;                  // cells [c0, c0 + ncell); c0 + ncell is the pad cell
    int n[3], nofs[3], ofs[3][kMaxStencil];
    int S;                          // segments per home cell (nofs_y * nofs_z)
    // rbl_obs constants of the replica, each rounded as written: 3N, V = (L_x L_y) L_z,
    // rho = N / V, 3V and the LJ tail terms at r_s (Sec. 3)
    double n3, V, rho, V3, U_tail, P_tail;
};

// Kernel-visible view of a context (passed by value).
//
// Neighbour storage.  All particles of a home cell share one candidate sequence:
// the members of the cells of its stencil in canonical order (stencil slots
// z-major, x-minor; members of a cell by x image, then tag).  Along x the stencil
// cells of one (y, z) offset are adjacent in memory, so the sequence is S_r =
// nofs_y * nofs_z "segments", each one contiguous run of particle indices, or two
// when it wraps around the periodic x face.  With pre_s the candidates before
// segment s and A, B its pieces, seg_tab[c][s] = (startA - pre_s, pre_s + lenA,
// startB - pre_s - lenA, pre_s + lenA + lenB): candidate k of the segment is particle
// k < .y ? .x + k : .z + k, and .w is the running count through the segment.  Rows
// are S = max_r S_r entries long; entries past the replica's S_r are (0, M_c, 0, M_c),
// so seg_tab[c][S-1].w = M_c for every cell.
// Shell sampling keeps, per home cell, the culled candidate table ctab[c][0..T_c):
// the candidate sequence without the candidates that no particle of the cell can
// reach (farther than r_s + skin, with a margin that covers every binary32 rounding
// of the pair rule, from the bounding box of the cell's particles at the build), in
// the same order.  A dropped candidate is in no row of the cell, so rows are the
// same whichever sequence the masks index.
// Per particle slot:
//   core  : explicit list of neighbour indices, column-major core[k][N];
//   shell : bitmask over the culled table, column-major mask[w][N], bit b of word w
//           <-> ctab entry 32 w + b (full_list mode: explicit rows in core instead).
// A shell row in canonical order is the table filtered by the mask, so the position
// of a neighbour in its row is its rank among the set bits.
struct View {
    int N;                          // particle slots of all replicas (stride of per-particle arrays)
    int R;                          // replicas
    int ntile;                      // N / kTile
    int p, K, cap_c, W, S, Mcap, full_list, precision, subtract;
    int sampling;                   // RBL_SAMPLE_SHELL or RBL_SAMPLE_STENCIL
    int potential;                  // RBL_POT_LJ or RBL_POT_LJ_EWALD
    float alpha32, ka32;            // Ewald alpha and 2 alpha / sqrt(pi), binary32
    double alpha, ka;               // the same in FP64
    int force_threads;              // threads per block of the force kernel (64, 128 or 256)
    int build_warps;                // home cells (warps) per block of the list build (2, 4 or 8)
    int ncell;                      // cells of all replicas, pad cells included
    float t_core_list, t_shell_lo, t_cut_list, t_rc2, t_rs2, t_disp;
    float t_cull;                   // (r_s + skin)^2 (1 + 2^-12): the list build's bounding-box cull
    double dt, gamma, c1;
    const Box *box;                 // [R]
    const int2 *tile;               // [ntile]: (replica, end of its live slots)
    const int *cell_rep;            // [ncell]: replica of each cell
    // state (cell order within each replica); [axis][N] for x and v
    double *x, *v;                  // current buffer base (3 consecutive N-arrays each)
    double *x_alt, *v_alt;          // other buffer (permutation target)
    int *tag, *tag_alt;             // tag = particle number within its replica
    int4 *pos, *pos_alt;            // (ux, uy, uz, tag) 32-bit fixed-point image
    int4 *ubuild;                   // image at the last build
    double *q;                      // charges in cell order (RBL_POT_LJ_EWALD; else null)
    float *q32;                     // the same in binary32 (FP32 pair arithmetic)
    double *q_in;                   // charges in load order: slot first + t holds tag t's
    void *F;                        // [3][N]: int64 fixed point (FP32 path) or double
    int *cell, *order;
    int *counts, *start, *fill, *blocksums;
    int4 *seg_tab;                  // [ncell][S]
    int *ctab;                      // [ncell][Mcap]: culled candidate table (shell sampling; Mcap
                                    // is its capacity, W = Mcap / 32 mask words)
    int *ctab_n;                    // [ncell]: its length T_c
    int *core, *n_core;             // core[k * N + i], k < cap_c
    unsigned *mask;                 // mask[w * N + i], w < W
    int *n_shell;                   // set bits in the mask (N_s, or full-list length)
    int *hcell;                     // home cell (global index) of each particle at the last build
    double *partials;               // [64-thread groups][8]
    double *partials2;              // [R][pchunks][8]: the groups' partials summed per chunk of 256
    int pchunks;                    // chunks of the largest replica
    RepScalars *rs;                 // [R]
    DevScalars *sc;
    double *staging;                // host/device I/O scratch
    unsigned long long *kin_acc;    // [8][kin_stride]: observables launch, replica r's sums of v^2,
                                    // v_x, v_y, v_z as (integer part, fraction in units of 2^-40), each
                                    // summed over tiles (mod 2^64); zero between launches
    int kin_stride;                 // R rounded up to 16 (one 128-byte line per value and 16 replicas)
};

// Replica of particle slot i (i < N) and whether the slot holds a particle.
__device__ __forceinline__ int slot_replica(const View &v, int i, bool &live)
{
    const int2 t = v.tile[i >> kTileShift];
    live = i < t.y;
    return t.x;
}

// Wrap a cell coordinate into [0, n) for -n <= c < 2n (stencil offsets never
// reach further): compare-and-add instead of an integer division.
__host__ __device__ __forceinline__ int wrap_cell(int c, int n)
{
    c = c >= n ? c - n : c;
    return c < 0 ? c + n : c;
}

// Streams the segments of a home cell in ascending candidate order and maps a
// candidate index to a particle index: one 16-byte table load per segment.
struct SegCursor {
    const int4 *tab;      // seg_tab row of the home cell
    int seg;              // current segment
    int4 e;               // its table entry

    __host__ __device__ __forceinline__ void init(const int4 *tabp)
    {
        tab = tabp;
        seg = 0;
        e = tab[0];
    }
    // cand must not decrease between calls.
    __host__ __device__ __forceinline__ int index_of(int cand)
    {
        while (cand >= e.w) e = tab[++seg];
        return cand < e.y ? e.x + cand : e.z + cand;
    }
};

// Stencil-pool sampling: the particle's own position in its home cell's candidate
// sequence (the pool is that sequence without it).  The home cell lies in the row
// of (y, z) offset 0: index m of the offsets -m..m, or 0 when every cell is visited
// once starting from the home cell.
__device__ __forceinline__ int pool_self_position(const Box &b, const int4 *tab, int i)
{
    const int iz = b.ofs[2][0] < 0 ? -b.ofs[2][0] : 0;
    const int iy = b.ofs[1][0] < 0 ? -b.ofs[1][0] : 0;
    const int s = iz * b.nofs[1] + iy;
    const int4 e = tab[s];
    const int pre = s > 0 ? tab[s - 1].w : 0;
    const int candA = i - e.x;
    return (candA >= pre && candA < e.y) ? candA : i - e.z;
}

// Position (0..31) of the r-th (0-based) set bit of w; w must have more than r bits.
__host__ __device__ __forceinline__ int select_bit(unsigned w, int r)
{
#ifdef __CUDA_ARCH__
#define RBL_POPC(x) __popc(x)
#else
#define RBL_POPC(x) __builtin_popcount(x)
#endif
    int pos = 0;
    int c = RBL_POPC(w & 0xFFFFu);
    if (r >= c) { r -= c; pos = 16; }
    c = RBL_POPC((w >> pos) & 0xFFu);
    if (r >= c) { r -= c; pos += 8; }
    c = RBL_POPC((w >> pos) & 0xFu);
    if (r >= c) { r -= c; pos += 4; }
    c = RBL_POPC((w >> pos) & 0x3u);
    if (r >= c) { r -= c; pos += 2; }
    c = (int)((w >> pos) & 1u);
    if (r >= c) pos += 1;
    return pos;
#undef RBL_POPC
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): published multipliers and
// Weyl key increments; ten rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Word stream for (seed, step, tag, stream): counter (step_lo, step_hi, tag,
// stream<<24 | block), four words per block consumed in order.
struct WordStream {
    uint32_t k0, k1, s0, s1, tag, blk;
    uint4 buf;
    int pos;
    __device__ __forceinline__ void init(unsigned long long seed, unsigned long long step, uint32_t t, uint32_t stream)
    {
        k0 = (uint32_t)seed;
        k1 = (uint32_t)(seed >> 32);
        s0 = (uint32_t)step;
        s1 = (uint32_t)(step >> 32);
        tag = t;
        blk = stream << 24;
        pos = 4;
    }
    __device__ __forceinline__ uint32_t next()
    {
        if (pos == 4) {
            buf = philox4x32_10(make_uint4(s0, s1, tag, blk), k0, k1);
            blk += 1u;
            pos = 0;
        }
        uint32_t w = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
        ++pos;
        return w;
    }
};

// Uniform integer in [0, s) (Lemire 2019, multiply-shift with rejection).  The
// rejection loop is capped; hitting the cap (probability below (s/2^32)^64) sets a
// flag instead of spinning.
__device__ __forceinline__ uint32_t uniform_below(WordStream &ws, uint32_t s, unsigned *flags)
{
    unsigned long long m = (unsigned long long)ws.next() * s;
    uint32_t low = (uint32_t)m;
    if (low < s) {
        uint32_t threshold = (0u - s) % s;
        int guard = 0;
        while (low < threshold) {
            if (++guard > 64) {
                atomicOr(flags, kFlagRngLimit);
                break;
            }
            m = (unsigned long long)ws.next() * s;
            low = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

// Floyd's sampling of p distinct positions in [0, ns) (Bentley & Floyd 1987), in
// draw order; when ns <= p every position is taken.  Returns the count.
__device__ __forceinline__ int floyd_positions(unsigned long long seed, unsigned long long step, int tag, int ns,
                                               int p, int *S, unsigned *flags)
{
    if (ns <= p) {
        for (int q = 0; q < ns; ++q) S[q] = q;
        return ns;
    }
    WordStream ws;
    ws.init(seed, step, (uint32_t)tag, 0u);
    for (int q = 0; q < p; ++q) {
        int k = ns - p + q;
        int t = (int)uniform_below(ws, (uint32_t)k + 1u, flags);
        bool seen = false;
        for (int r = 0; r < q; ++r) seen |= (S[r] == t);
        S[q] = seen ? k : t;
    }
    return p;
}

// Register-resident batch for p <= PMAX: the Floyd positions, kept sorted ascending
// while they are drawn and padded with INT_MAX; returns min(N_s, p).  Floyd's step q
// either inserts t (uniform in [0, k]) or, when t is already taken, k itself -- and k
// exceeds every earlier pick, so it lands at the end.  One pass of compares against
// the sorted prefix gives both "already taken" and t's insertion point.
// Fast path: draw q uses word q of the stream.  A draw whose low word lies below its
// bound could be rejected by Lemire's rule and would shift the stream; the batch is
// then redrawn by floyd_positions (the general sampler) and sorted, so both paths
// give identical batches.
template <int PMAX>
__device__ __forceinline__ int batch_sorted(unsigned long long seed, unsigned long long step, int tag, int ns,
                                            int p, int (&S)[PMAX], unsigned *flags)
{
    const int kInf = 0x7fffffff;
#pragma unroll
    for (int q = 0; q < PMAX; ++q) S[q] = kInf;
    if (ns <= p) {
#pragma unroll
        for (int q = 0; q < PMAX; ++q) S[q] = q < ns ? q : kInf;
        return ns;
    }
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c0 = (uint32_t)step, c1 = (uint32_t)(step >> 32);
    bool slow = false;
    uint4 blk = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
        if (q < p) {
            if ((q & 3) == 0) blk = philox4x32_10(make_uint4(c0, c1, (uint32_t)tag, (uint32_t)(q >> 2)), k0, k1);
            const uint32_t w = (q & 3) == 0 ? blk.x : (q & 3) == 1 ? blk.y : (q & 3) == 2 ? blk.z : blk.w;
            const uint32_t bound = (uint32_t)(ns - p + q) + 1u;
            const unsigned long long m = (unsigned long long)w * bound;
            slow |= (uint32_t)m < bound;
            const int t = (int)(m >> 32);
            bool seen = false;
            int pos = 0;
#pragma unroll
            for (int r = 0; r < q; ++r) {
                seen |= S[r] == t;
                pos += S[r] < t ? 1 : 0;
            }
            const int x = seen ? (int)(bound - 1u) : t;
            if (seen) pos = q;
            // insert x at pos into the sorted prefix S[0..q)
#pragma unroll
            for (int r = q; r > 0; --r) S[r] = r > pos ? S[r - 1] : (r == pos ? x : S[r]);
            S[0] = pos == 0 ? x : S[0];
        }
    }
    if (slow) {
        int T[kMaxP];
        const int nb = floyd_positions(seed, step, tag, ns, p, T, flags);
        for (int a = 1; a < nb; ++a) { // insertion sort (rare path)
            int x = T[a], b = a - 1;
            while (b >= 0 && T[b] > x) {
                T[b + 1] = T[b];
                --b;
            }
            T[b + 1] = x;
        }
#pragma unroll
        for (int q = 0; q < PMAX; ++q) S[q] = q < nb ? T[q] : kInf;
    }
    return p;
}

// ---------------------------------------------------------------------------
// Canonical pair rule: d = (float)(int32)(u_i - u_j) * h, r2 = (dx dx + dy dy) + dz dz,
// every operation rounded separately.
// ---------------------------------------------------------------------------
struct PairGeom {
    float dx, dy, dz, r2;
};

__device__ __forceinline__ PairGeom pair_geom(int4 a, int4 b, const float h[3])
{
    PairGeom g;
    g.dx = __fmul_rn(__int2float_rn((int)((unsigned)a.x - (unsigned)b.x)), h[0]);
    g.dy = __fmul_rn(__int2float_rn((int)((unsigned)a.y - (unsigned)b.y)), h[1]);
    g.dz = __fmul_rn(__int2float_rn((int)((unsigned)a.z - (unsigned)b.z)), h[2]);
    g.r2 = __fadd_rn(__fadd_rn(__fmul_rn(g.dx, g.dx), __fmul_rn(g.dy, g.dy)), __fmul_rn(g.dz, g.dz));
    return g;
}

// Cell coordinate along one axis: floor(u n / 2^32), exact.
__device__ __forceinline__ int cell_coord(unsigned u, int n)
{
    return (int)(((unsigned long long)u * (unsigned)n) >> 32);
}

// LJ 12-6 in binary32: returns the force coefficient fmag with f = fmag * d, and
// the pair energy / virial when asked.  1/r^2 comes from the hardware reciprocal
// (rcp.approx, within 1 ulp); every path that must agree bit for bit (RBL with the
// whole shell, the full list) goes through this same function.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lj_coef(float r2, float *u, float *w)
{
    float inv = rcp_approx(r2);
    float r6 = __fmul_rn(__fmul_rn(inv, inv), inv);
    float t = __fmaf_rn(2.0f, r6, -1.0f);         // 2 r^-6 - 1
    float vir = __fmul_rn(__fmul_rn(24.0f, r6), t); // 24 (2 r^-12 - r^-6) = r . f
    if (u) *u = __fmul_rn(__fmul_rn(4.0f, r6), __fadd_rn(r6, -1.0f));
    if (w) *w = vir;
    return __fmul_rn(vir, inv);
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// LJ plus the Ewald real-space term in binary32: u = 4 (r^-12 - r^-6) + qq erfc(alpha
// r) / r and r . f = 24 (2 r^-12 - r^-6) + qq (erfc(alpha r) / r + ka exp(-alpha^2
// r^2)), ka = 2 alpha / sqrt(pi); returns the force coefficient (r . f) / r^2.  The
// LJ terms are formed exactly as in lj_coef.  erfc(x) = t h(t) exp(-x^2) with
// t = 1 / (1 + P x) and h the fitted polynomial of rbl_erfc_fit.cuh (relative error
// about 1e-7), so the one exponential serves both terms; 1/r, the reciprocal and
// 2^x come from the hardware approximations (within 2 ulp).
__device__ __forceinline__ float lj_ewald_coef(float r2, float qq, float alpha, float ka, float *u, float *w)
{
    float inv = rcp_approx(r2);
    float r6 = __fmul_rn(__fmul_rn(inv, inv), inv);
    float t = __fmaf_rn(2.0f, r6, -1.0f);
    float vlj = __fmul_rn(__fmul_rn(24.0f, r6), t);
    const float ir = rsqrt_approx(r2);                           // 1 / r
    const float ar = __fmul_rn(alpha, __fmul_rn(r2, ir));        // alpha r
    const float tt = rcp_approx(__fmaf_rn(kErfcP, ar, 1.0f));
    float hp = erfc_fit_coef(kErfcDegree);
#pragma unroll
    for (int k = kErfcDegree - 1; k >= 0; --k) hp = __fmaf_rn(hp, tt, erfc_fit_coef(k));
    const float ex = ex2_approx(__fmul_rn(__fmul_rn(ar, ar), -1.44269504f)); // exp(-alpha^2 r^2)
    const float ec = __fmul_rn(__fmul_rn(__fmul_rn(tt, hp), ex), ir);       // erfc(alpha r) / r
    const float vir = __fadd_rn(vlj, __fmul_rn(qq, __fmaf_rn(ka, ex, ec)));
    if (u) *u = __fadd_rn(__fmul_rn(__fmul_rn(4.0f, r6), __fadd_rn(r6, -1.0f)), __fmul_rn(qq, ec));
    if (w) *w = vir;
    return __fmul_rn(vir, inv);
}

// ---------------------------------------------------------------------------
// Exact fixed-point accumulation of binary32 values at scale 2^24.  Each value f
// with |f| < 2^20 is split without rounding error into A = rint(4f) and
// B = rint((4f - A) 2^22), so rint(f 2^24) = A 2^22 + B; A and B are summed as
// 32-bit integers (order-independent, exact), using the 1.5 * 2^23 bias trick so
// that both conversions are single binary32 operations.  For 2^20 <= |f| < 2^29
// (nearly overlapping pairs) the same split is taken with exact integer
// conversions (4f - rint(4f) is 0 or 1/2 there).
// ---------------------------------------------------------------------------
struct FixedAcc {
    unsigned a[3], b[3];
    int n;
    __device__ __forceinline__ void zero()
    {
        a[0] = a[1] = a[2] = b[0] = b[1] = b[2] = 0u;
        n = 0;
    }
    __device__ __forceinline__ void add1_small(int k, float f)
    {
        const float M = 12582912.0f; // 1.5 * 2^23
        float y = __fmaf_rn(f, 4.0f, M);
        float hpart = __fsub_rn(y, M);
        float r = __fmaf_rn(f, 4.0f, -hpart);
        float z = __fmaf_rn(r, 4194304.0f, M);
        a[k] += __float_as_uint(y);
        b[k] += __float_as_uint(z);
    }
    __device__ __forceinline__ void add1_large(int k, float f)
    {
        const unsigned bias = 0x4B400000u;
        float g = fminf(fmaxf(__fmul_rn(f, 4.0f), -2147483520.0f), 2147483520.0f);
        float y = rintf(g);                      // exact
        float r = __fsub_rn(g, y);               // 0 or +-1/2, exact
        a[k] += (unsigned)__float2int_rn(y) + bias;
        b[k] += (unsigned)__float2int_rn(__fmul_rn(r, 4194304.0f)) + bias;
    }
    // m: an upper bound of max(|fx|, |fy|, |fz|)
    __device__ __forceinline__ void add(float fx, float fy, float fz, float m)
    {
        if (m < 1048576.0f) {
            add1_small(0, fx);
            add1_small(1, fy);
            add1_small(2, fz);
        } else {
            add1_large(0, fx);
            add1_large(1, fy);
            add1_large(2, fz);
        }
        ++n;
    }
    // Exact int64 value of the sum at scale 2^24 for component k.
    __device__ __forceinline__ long long value(int k) const
    {
        const unsigned bias = 0x4B400000u; // bit pattern of 1.5 * 2^23
        int A = (int)(a[k] - (unsigned)n * bias);
        int B = (int)(b[k] - (unsigned)n * bias);
        return (long long)A * 4194304LL + (long long)B;
    }
};

constexpr double kFixedScale = 16777216.0;          // 2^24
constexpr double kFixedInv = 1.0 / 16777216.0;

// binary32 -> FP64 by bit manipulation (normal numbers and zero; subnormals -> 0).
__device__ __forceinline__ double f32_to_double(float f)
{
    unsigned b = __float_as_uint(f);
    unsigned e = (b >> 23) & 0xffu;
    unsigned long long r = (unsigned long long)(b >> 31) << 63;
    if (e != 0u)
        r |= ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)r);
}

// Fixed-point image of a coordinate x in [0, L): rint(x * 2^32/L) mod 2^32 with a
// single rounding: one fused multiply-add onto 1.5 * 2^52, whose ulp is 1, rounds
// the exact product to the nearest integer (ties to even).
__device__ __forceinline__ unsigned quantize(double x, double inv)
{
    const double y = __fma_rn(x, inv, 6755399441055744.0);
    return (unsigned)(unsigned long long)__double_as_longlong(y);
}

// Wrap into [0, L) for a particle that moved by less than L.  The comparisons are
// done on the IEEE bit patterns (integer units) instead of the FP64 pipe: for
// x >= 0 the order of the patterns is the order of the values.
__device__ __forceinline__ double wrap(double x, double L)
{
    long long b = __double_as_longlong(x);
    if (b < 0) {                 // sign bit: x < 0 (or -0.0)
        x += L;
        b = __double_as_longlong(x);
    }
    if (b >= __double_as_longlong(L)) x -= L;
    return x;
}

// 0 <= x < L for finite x and L > 0, from the IEEE bit patterns: a negative x has
// the sign bit set (a negative int64), and for x >= 0 the patterns order as the values.
__device__ __forceinline__ bool in_box_bits(double x, double L)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 && b < __double_as_longlong(L);
}

// Not NaN/inf, from the exponent bits.
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7FF0000000000000ull) != 0x7FF0000000000000ull;
}

inline int ceil_div(long long a, int b) { return (int)((a + b - 1) / b); }

} // namespace rbl

// Host-side context (C ABI handle).
struct rbl_ctx {
    rbl_params prm;              // replica 0's parameters (the shared ones are equal for all)
    rbl::View view;
    cudaStream_t stream;
    int R;                       // replicas
    long long n_real;            // particles of all replicas (rows of the packed caller arrays)
    int n_scan_blocks;
    int lists_valid;   // lists match the current positions
    int force_valid;   // F matches the current positions and step counter
    int energy_valid;  // energy/virial estimates match F
    int kick_pending;  // the last step call's closing half kick (dt/2 F) is not applied yet
    long long step;    // host mirror of the step counter
    size_t staging_bytes;
    cudaGraphExec_t graph_exec[4]; // captured steps: middle, first, last, single (enum StepGraph)
    int phase_timing;           // rbl_set_phase_timing
    cudaEvent_t *ev;            // kPhaseEvents events per timed step
    int ev_cap;                 // steps the event pool covers
    double phase_ms[5];
    long long phase_steps;
    double rebuild_ms[2];       // phase timing: forced rebuilds' cell sort chain and list build
    long long rebuild_n;        // forced rebuilds timed
    cudaEvent_t rb_ev[3];       // their events (created on first use)
    char err[512];
    rbl::DevScalars *h_sc;      // host mirror of the device scalars
    rbl::RepScalars *h_rs;      // host mirror of the per-replica scalars [R]
    rbl::Box *h_box;            // host copy of the replica table [R]
    int2 *h_tile;               // host copy of the tile table [ntile]
    int *h_cell_rep;            // host copy of the cell -> replica table [ncell]
};

// Kernel launchers implemented in the .cu files.
namespace rbl {
cudaError_t launch_load_state(const View &v, const double *x, const double *vel, cudaStream_t s);
// ck: a half kick still pending at the end of a step call, applied to the velocities
// written (or summed) but not to the state
cudaError_t launch_store_state(const View &v, double *x, double *vel, cudaStream_t s, double ck = 0.0);
cudaError_t launch_store_images(const View &v, unsigned *img, cudaStream_t s);
cudaError_t launch_load_images(const View &v, const unsigned *img, cudaStream_t s);
cudaError_t launch_requantize(const View &v, cudaStream_t s);
cudaError_t launch_rebuild(const View &v, int n_scan_blocks, bool conditional, cudaStream_t s);
// the two halves of launch_rebuild: cell hash, scan, sort and permutation; then the lists
cudaError_t launch_rebuild_sort(const View &v, int n_scan_blocks, bool conditional, cudaStream_t s);
cudaError_t launch_rebuild_lists(const View &v, bool conditional, cudaStream_t s);
cudaError_t launch_set_rebuild_condition(const View &v, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t launch_forces(const View &v, int step_offset, int advance, bool energy, cudaStream_t s);
// prepare = true: set the kernel's attributes for a later captured launch, launch nothing
cudaError_t launch_force_kernel(const View &v, int step_offset, bool energy, cudaStream_t s, bool prepare = false);
cudaError_t launch_force_finish(const View &v, int advance, bool energy, cudaStream_t s);
cudaError_t launch_init_single(const View &v, const Box &b, cudaStream_t s);
cudaError_t launch_exact_energy(const View &v, cudaStream_t s);
cudaError_t launch_store_forces(const View &v, double *F, cudaStream_t s);
cudaError_t launch_integrate(const View &v, double ck, bool drift, cudaStream_t s);
cudaError_t launch_observables(const View &v, rbl_obs *out, double ck, cudaStream_t s);
cudaError_t launch_batch(const View &v, unsigned long long step, int *out_j, int *out_n, cudaStream_t s);
cudaError_t launch_rdf(const View &v, float dr, int nbins, unsigned long long *hist, cudaStream_t s);
cudaError_t launch_profile(const View &v, int axis, int nbins, unsigned long long *hist, cudaStream_t s);
cudaError_t launch_set_charges(const View &v, const double *q_packed, cudaStream_t s);
// The force kernel with the LJ + Ewald real-space pair (its own translation unit).
cudaError_t launch_force_kernel_ewald(const View &v, int step_offset, bool energy, cudaStream_t s, bool prepare);
cudaError_t launch_exact_energy_kernel_ewald(const View &v, cudaStream_t s);
constexpr int kMaxProfileBins = 12288; // shared-memory histogram of one block
} // namespace rbl
