// rbl_force_kernel.cuh -- the force kernel of the RBL (Sec. 2, Eqs. (3)-(4)) and of
// the classical full list, templated on the pair potential; rbl_force.cu
// instantiates it for LJ and rbl_force_ewald.cu for LJ plus the Ewald real-space
// term, in parallel translation units.
//
// One thread per particle (cell order).  Core row: every entry with r < r_c is
// summed.  Shell: a Floyd p-subset of positions is drawn from Philox stream 0 of
// (seed, step, tag) -- or everything when N <= p -- sorted, and each drawn position
// is mapped to its neighbour: in the shell mask by its rank among the set bits
// (shell sampling), or directly in the home cell's stencil (the paper's stencil
// pool).  Every drawn neighbour with r_c <= r < r_s contributes s f_ij, s = N / p.
// The mask words are read column-major, so a warp reads 32 consecutive particles'
// words in one transaction.
//
// FP32 path: pair arithmetic in binary32, the core and batch terms summed per
// particle in binary32 in the canonical order, the total converted once, exactly,
// to int64 fixed point at scale 2^24, so sums over particles are exact and do not
// depend on order or thread mapping.  FP64 path: FP64 pair arithmetic from the FP64
// positions, per-64-thread partial sums reduced in a fixed order.
#pragma once

#include "rbl_internal.cuh"

namespace rbl {

namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Deterministic partial sums of NV doubles per thread, one partial per 64-thread
// group whatever the block size (64, 128 or 256): warp sums by a fixed shuffle
// tree, then the group's two warps in order, into partials[group][off..off+NV).
// The reductions built on them therefore do not depend on the launch shape.
constexpr int kMaxForceThreads = 256;
template <int NV>
__device__ __forceinline__ void group_sums(double (&x)[NV], double *partials, int off)
{
    __shared__ double sh[NV][kMaxForceThreads / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, ng = blockDim.x >> 6;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(x[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if ((int)threadIdx.x < NV * ng) {
        const int g = threadIdx.x / NV, k = threadIdx.x - g * NV;
        const size_t group = (size_t)blockIdx.x * ng + g;
        partials[group * 8 + off + k] = sh[k][2 * g] + sh[k][2 * g + 1];
    }
}

// Per-particle accumulators.  FP32 path: binary32 pair terms summed in binary32 in
// the canonical order (core row order, then the batch in ascending row position),
// the shell sum scaled by s once; the per-particle total is converted exactly to
// int64 fixed point (scale 2^24) for every cross-particle sum.  FP64 path: FP64
// pair terms from the FP64 positions.
template <bool FP32, bool ENERGY, bool EWALD>
struct Accum {
    float f32[2][3], e32[2], w32[2];   // [0] core, [1] shell (before the batch scale)
    double f64[2][3], e64[2], w64[2];
    float h[3];                        // the replica's fixed-point unit L / 2^32
    const double *L;                   // the replica's box (FP64 path)
    float qi32;                        // the particle's charge (EWALD)
    double qi64;

    __device__ __forceinline__ void zero(const Box &b)
    {
        h[0] = b.h[0];
        h[1] = b.h[1];
        h[2] = b.h[2];
        L = b.L;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                f32[r][a] = 0.f;
                f64[r][a] = 0.0;
            }
            e32[r] = w32[r] = 0.f;
            e64[r] = w64[r] = 0.0;
        }
    }

    __device__ __forceinline__ static bool in_region(const View &v, float r2, int part)
    {
        if (v.full_list) return r2 < v.t_rs2;
        return part == 0 ? r2 < v.t_rc2 : (r2 >= v.t_rc2 && r2 < v.t_rs2);
    }

    __device__ __forceinline__ void set_charge(const View &v, int i)
    {
        if constexpr (EWALD) {
            if (FP32) qi32 = v.q32[i];
            else qi64 = v.q[i];
        }
    }

    // Pair (i, j) in region `part` (0 core, 1 shell / full); qj32 / qj64: the
    // neighbour's charge (EWALD).
    __device__ __forceinline__ void pair(const View &v, int4 pi, int4 pj, int i, int j, int part, float qj32,
                                         double qj64)
    {
        PairGeom g = pair_geom(pi, pj, h);
        bool inside = in_region(v, g.r2, part);
        if (FP32) {
            float u, w, coef;
            if constexpr (EWALD)
                coef = lj_ewald_coef(g.r2, __fmul_rn(qi32, qj32), v.alpha32, v.ka32, &u, &w);
            else
                coef = lj_coef(g.r2, &u, &w);
            coef = inside ? coef : 0.f;
            f32[part][0] = __fmaf_rn(coef, g.dx, f32[part][0]);
            f32[part][1] = __fmaf_rn(coef, g.dy, f32[part][1]);
            f32[part][2] = __fmaf_rn(coef, g.dz, f32[part][2]);
            if (ENERGY && inside) {
                e32[part] += u;
                w32[part] += w;
            }
        } else if (inside) {
            size_t N = (size_t)v.N;
            double d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double t = v.x[a * N + i] - v.x[a * N + j];
                t -= L[a] * rint(t / L[a]);
                d[a] = t;
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double inv = 1.0 / r2;
            double r6 = inv * inv * inv;
            double vir = 24.0 * (2.0 * r6 * r6 - r6);
            double e = 4.0 * (r6 * r6 - r6);
            if constexpr (EWALD) {
                // q_i q_j erfc(alpha r) / r and its virial (erfc, exp: CUDA's FP64 functions)
                const double qq = qi64 * qj64;
                const double r = sqrt(r2);
                const double ar = v.alpha * r;
                const double ec = erfc(ar) / r;
                e += qq * ec;
                vir += qq * (ec + v.ka * exp(-ar * ar));
            }
            double coef = vir * inv;
#pragma unroll
            for (int a = 0; a < 3; ++a) f64[part][a] += coef * d[a];
            e64[part] += e;
            w64[part] += vir;
        }
    }

    // kGather pairs: indices jj[u] (valid for u < cnt), gathered before any is used.
    template <int G>
    __device__ __forceinline__ void pairs(const View &v, int4 pi, int i, const int (&jj)[G], int cnt, int part)
    {
        int4 pj[G];
        float q32[G];
        double q64[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int j = u < cnt ? jj[u] : i;
            pj[u] = v.pos[j];
            if constexpr (EWALD) {
                if (FP32) q32[u] = v.q32[j];
                else q64[u] = v.q[j];
            } else {
                q32[u] = 0.f;
                q64[u] = 0.0;
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u)
            if (u < cnt) pair(v, pi, pj[u], i, jj[u], part, FP32 ? q32[u] : 0.f, FP32 ? 0.0 : q64[u]);
    }
};

__device__ __forceinline__ void sort_small(int *S, int n)
{
    for (int a = 1; a < n; ++a) {
        int x = S[a], b = a - 1;
        while (b >= 0 && S[b] > x) {
            S[b + 1] = S[b];
            --b;
        }
        S[b + 1] = x;
    }
}

// EWALD: the pair is LJ plus the Ewald real-space term q_i q_j erfc(alpha r) / r.
// MODE 0: RBL (core list + sampled shell mask); MODE 1: full list (explicit rows);
// MODE 2: exact observables -- the core list and every shell (or full) mask entry,
// or every pool member, unsampled, energy and virial only (no force written, no
// total force); MODE 3: RBL with the batch drawn from the stencil pool.
// PMAX > 0: batch positions and neighbour indices live in registers (p <= PMAX);
// PMAX = 0: general path through local arrays (p up to kMaxP).
//
// Memory-level parallelism: the mask words of a thread are staged in shared memory
// with bursts of independent loads (column-major storage makes every burst coalesced
// across the warp), the batch is drawn while those loads are in flight, and
// neighbour indices and positions are gathered `gather` at a time before their pair
// terms are computed.
// Threads per block: a launch parameter of the context (64, 128 or 256; chosen by
// rbl_autotune); the staging arrays are dynamic shared memory sized for the block.
static_assert(kMinBlock == 64 && kMaxForceThreads % 64 == 0, "per-block partials are sized for kMinBlock");
constexpr int kMaskStage = 32;  // mask words staged per thread (longer rows read directly)
// the rank search halves its step from kMaskStage / 2, so it reaches every staged word
// only for a power of two
static_assert(kMaskStage > 0 && (kMaskStage & (kMaskStage - 1)) == 0 && kMaskStage <= 32,
              "kMaskStage must be a power of two no larger than 32");

// Gather width and FP32 register cap per mode, measured on GB300 (the LJ fluid and
// the charged fluid at N = 2^20, best block shape of each): shell sampling runs
// fastest with 4 gathers in flight and 64 registers (4 blocks of 256 threads per SM),
// the stencil pool with 12 and 80 (8 and 80 with the Ewald term), the full list's
// explicit rows with 8 and 80 (0.61 -> 0.53 ms; 16 and 128: 0.52 ms); the energy
// variants (last step of a call, one-step calls) keep their energy and virial sums in
// 72.  The FP64 path needs up to 128 registers and runs at the FP64 rate anyway.
// The full list's rows hold a multiple of 8 entries, so its 16-byte index loads stay
// inside a row.
template <int MODE, bool ENERGY, bool EWALD>
struct ForceTuning {
    static constexpr int gather = MODE == 1 ? 8 : (MODE == 3 ? (EWALD ? 8 : 12) : 4);
    static constexpr int regs = (MODE == 1 || MODE == 3) ? 80 : 64;
};

template <int MODE, bool FP32, bool ENERGY, int PMAX, bool EWALD>
__global__ void __maxnreg__((FP32 ? ForceTuning<MODE, ENERGY, EWALD>::regs : 128)) k_force(View v, int step_offset)
{
    constexpr int kGather = ForceTuning<MODE, ENERGY, EWALD>::gather;
    // staged mask words [kMaskStage][blockDim] and the set bits before each of them
    extern __shared__ unsigned s_dyn[];
    const int bd = blockDim.x;
    unsigned *s_mask = s_dyn;
    unsigned short *s_pref = (unsigned short *)(s_dyn + kMaskStage * bd);
    const unsigned long long step = v.sc->step + (unsigned long long)step_offset;
    const int t = threadIdx.x;
    const int i = blockIdx.x * bd + t;
    const size_t N = (size_t)v.N;
    long long qv[3] = {0, 0, 0};
    long long eq = 0, wq = 0;       // FP32 path, ENERGY: fixed-point energy and virial
    double f64[3] = {0.0, 0.0, 0.0};
    double e_i = 0.0, w_i = 0.0;
    bool live = false;
    const int r = i < v.N ? slot_replica(v, i, live) : 0;
    if (live) {
        const Box &b = v.box[r];
        const int4 pi = v.pos[i];
        const int nc = (MODE == 0 || MODE == 3 || (MODE == 2 && !v.full_list)) ? min(v.n_core[i], v.cap_c) : 0;
        const int ns = v.n_shell[i];
        const int hc = v.hcell[i];
        const int4 *tab = v.seg_tab + (size_t)hc * v.S;
        // shell sampling: the masks index the home cell's culled candidate table
        const int *ctab = v.ctab + (size_t)hc * v.Mcap;
        const int nwords = v.W > 0 ? min((v.ctab_n[hc] + 31) >> 5, v.W) : 0;
        // stage the mask words (independent loads, in bursts) and their running
        // popcounts
        const int nws = min(nwords, kMaskStage);
        int run = 0;
        for (int w0 = 0; w0 < nws; w0 += 8) {
            unsigned tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) tmp[u] = w0 + u < nws ? v.mask[(size_t)(w0 + u) * N + i] : 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (w0 + u < nws) {
                    s_mask[(w0 + u) * bd + t] = tmp[u];
                    s_pref[(w0 + u) * bd + t] = (unsigned short)run;
                    run += __popc(tmp[u]);
                }
        }
        auto mask_word = [&](int w) -> unsigned {
            return w < kMaskStage ? s_mask[w * bd + t] : v.mask[(size_t)w * N + i];
        };
        Accum<FP32, ENERGY, EWALD> acc;
        acc.zero(b);
        acc.set_charge(v, i);
        SegCursor cur;
        cur.init(tab);
        float s32 = 1.0f;
        double s64 = 1.0;
        if (MODE == 0) {
            // shell batch: positions in the row -> particle indices
            if constexpr (PMAX > 0) {
                int S[PMAX];
                const int nb = batch_sorted<PMAX>(b.seed, step, pi.w, ns, v.p, S, &v.sc->flags);
                if (ns > v.p) {
                    s32 = __fdiv_rn((float)ns, (float)v.p);
                    s64 = (double)ns / (double)v.p;
                }
                int J[PMAX];
                if (nwords <= kMaskStage) {
                    // Each drawn rank is resolved on its own, with no branch: the word
                    // holding it by a binary search over the staged running popcounts,
                    // the bit by select_bit, the particle by one load from the culled
                    // candidate table.  PMAX equals p (or bounds it), so the PMAX
                    // independent chains overlap; a data-dependent walk along the row
                    // would diverge across the warp and serialise them.  Slots past the
                    // batch resolve a clamped rank (an entry of the table's row) and are
                    // not used.
#pragma unroll
                    for (int q = 0; q < PMAX; ++q) {
                        const int tq = min(S[q], max(ns - 1, 0));
                        int w = 0;
#pragma unroll
                        for (int sw = kMaskStage / 2; sw >= 1; sw >>= 1) {
                            const int mid = w + sw;
                            const int pm = (int)s_pref[min(mid, kMaskStage - 1) * bd + t];
                            w = (mid < nws && pm <= tq) ? mid : w;
                        }
                        const int cand = (w << 5) + select_bit(s_mask[w * bd + t], tq - (int)s_pref[w * bd + t]);
                        J[q] = __ldg(&ctab[cand]);
                    }
                } else {
                    // rows longer than the staging area: walk the row in order
                    int w = 0, seen = 0;
                    unsigned word = nb > 0 ? mask_word(0) : 0u;
                    int cnt = __popc(word);
#pragma unroll
                    for (int q = 0; q < PMAX; ++q) {
                        J[q] = i;
                        if (q < nb) {
                            const int tq = S[q];
                            while (tq >= seen + cnt) {
                                seen += cnt;
                                word = mask_word(++w);
                                cnt = __popc(word);
                            }
                            J[q] = ctab[(w << 5) + select_bit(word, tq - seen)];
                        }
                    }
                }
#pragma unroll
                for (int q0 = 0; q0 < PMAX; q0 += kGather) {
                    if (q0 < nb) {
                        int jj[kGather];
#pragma unroll
                        for (int u = 0; u < kGather; ++u) // slots past the batch: unused
                            jj[u] = q0 + u < PMAX ? J[q0 + u] : i;
                        acc.template pairs<kGather>(v, pi, i, jj, nb - q0, 1);
                    }
                }
            } else {
                int S[kMaxP];
                const int nb = floyd_positions(b.seed, step, pi.w, ns, v.p, S, &v.sc->flags);
                if (ns > v.p) {
                    s32 = __fdiv_rn((float)ns, (float)v.p);
                    s64 = (double)ns / (double)v.p;
                    sort_small(S, nb);
                }
                int w = 0, seen = 0;
                unsigned word = nb > 0 ? mask_word(0) : 0u;
                int cnt = __popc(word);
                for (int q0 = 0; q0 < nb; q0 += kGather) {
                    int jj[kGather];
#pragma unroll
                    for (int u = 0; u < kGather; ++u) {
                        jj[u] = i;
                        if (q0 + u < nb) {
                            const int tq = S[q0 + u];
                            while (tq >= seen + cnt) {
                                seen += cnt;
                                word = mask_word(++w);
                                cnt = __popc(word);
                            }
                            jj[u] = ctab[(w << 5) + select_bit(word, tq - seen)];
                        }
                    }
                    acc.template pairs<kGather>(v, pi, i, jj, nb - q0, 1);
                }
            }
        }
        if (MODE == 3) {
            // stencil pool: rank t of the pool is candidate t (t + 1 past the particle's
            // own position) of the home cell's sequence; no masks
            const int self = pool_self_position(b, tab, i);
            if (ns > v.p) {
                s32 = __fdiv_rn((float)ns, (float)v.p);
                s64 = (double)ns / (double)v.p;
            }
            if constexpr (PMAX > 0) {
                int S[PMAX];
                const int nb = batch_sorted<PMAX>(b.seed, step, pi.w, ns, v.p, S, &v.sc->flags);
                int J[PMAX];
                const int S_ = v.S;
                const int top = S_ <= 32 ? 16 : 32;
#pragma unroll
                for (int q = 0; q < PMAX; ++q) {
                    const int tq = min(S[q], max(ns - 1, 0));
                    const int cand = tq + (tq >= self ? 1 : 0);
                    int sg = 0;
#pragma unroll
                    for (int sw = 32; sw >= 1; sw >>= 1) {
                        if (sw > top) continue;
                        const int m2 = sg + sw;
                        const int end = __ldg(&tab[min(m2, S_) - 1].w);
                        sg = (m2 <= S_ && end <= cand) ? m2 : sg;
                    }
                    const int4 e = __ldg(&tab[min(sg, S_ - 1)]);
                    J[q] = cand < e.y ? e.x + cand : e.z + cand;
                }
#pragma unroll
                for (int q0 = 0; q0 < PMAX; q0 += kGather) {
                    if (q0 < nb) {
                        int jj[kGather];
#pragma unroll
                        for (int u = 0; u < kGather; ++u) // slots past the batch: unused
                            jj[u] = q0 + u < PMAX ? J[q0 + u] : i;
                        acc.template pairs<kGather>(v, pi, i, jj, nb - q0, 1);
                    }
                }
            } else {
                int S[kMaxP];
                const int nb = floyd_positions(b.seed, step, pi.w, ns, v.p, S, &v.sc->flags);
                if (ns > v.p) sort_small(S, nb);
                for (int q0 = 0; q0 < nb; q0 += kGather) {
                    int jj[kGather];
#pragma unroll
                    for (int u = 0; u < kGather; ++u) {
                        jj[u] = i;
                        if (q0 + u < nb) {
                            const int tq = S[q0 + u];
                            jj[u] = cur.index_of(tq + (tq >= self ? 1 : 0));
                        }
                    }
                    acc.template pairs<kGather>(v, pi, i, jj, nb - q0, 1);
                }
            }
        }
        // core row, kGather at a time
        for (int k0 = 0; k0 < nc; k0 += kGather) {
            int jj[kGather];
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
                const int k = k0 + u;
                jj[u] = k < nc ? v.core[(size_t)k * N + i] : i;
            }
            acc.template pairs<kGather>(v, pi, i, jj, nc - k0, 0);
        }
        if (MODE == 2 && v.sampling) {
            // every pool member (the home cell's stencil less the particle itself)
            const int self = pool_self_position(b, tab, i);
            const int M = tab[v.S - 1].w;
            for (int c0 = 0; c0 < M; c0 += kGather) {
                int jj[kGather];
#pragma unroll
                for (int u = 0; u < kGather; ++u) {
                    const int c = c0 + u;
                    jj[u] = (c < M && c != self) ? cur.index_of(c) : i;
                }
                acc.template pairs<kGather>(v, pi, i, jj, min(kGather, M - c0), 1);
            }
        } else if ((MODE == 1 || MODE == 2) && v.full_list) {
            // the full list's explicit row (row-major, cap_c entries of which the first
            // n are set), kGather members at a time; four indices per 16-byte load
            const int *row = v.core + (size_t)i * (size_t)v.cap_c;
            const int n = min(ns, v.cap_c);
            for (int k0 = 0; k0 < n; k0 += kGather) {
                int jj[kGather];
                if constexpr (kGather % 4 == 0) {
#pragma unroll
                    for (int u = 0; u < kGather; u += 4) {
                        const int4 e = __ldg((const int4 *)(row + k0 + u));
                        jj[u] = k0 + u < n ? e.x : i;
                        jj[u + 1] = k0 + u + 1 < n ? e.y : i;
                        jj[u + 2] = k0 + u + 2 < n ? e.z : i;
                        jj[u + 3] = k0 + u + 3 < n ? e.w : i;
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < kGather; ++u) jj[u] = k0 + u < n ? row[k0 + u] : i;
                }
                acc.template pairs<kGather>(v, pi, i, jj, n - k0, 1);
            }
        } else if (MODE == 2) {
            // every shell mask entry, kGather members at a time
            int w = 0;
            unsigned word = ns > 0 ? mask_word(0) : 0u;
            for (int k0 = 0; k0 < ns; k0 += kGather) {
                int jj[kGather];
#pragma unroll
                for (int u = 0; u < kGather; ++u) {
                    jj[u] = i;
                    if (k0 + u < ns) {
                        while (word == 0u) word = mask_word(++w);
                        const int bit = __ffs(word) - 1;
                        word &= word - 1u;
                        jj[u] = ctab[(w << 5) + bit];
                    }
                }
                acc.template pairs<kGather>(v, pi, i, jj, ns - k0, 1);
            }
        }
        if (MODE == 2) {
            if (FP32) {
                e_i = 0.5 * ((double)acc.e32[0] + (double)acc.e32[1]);
                w_i = 0.5 * ((double)acc.w32[0] + (double)acc.w32[1]);
            } else {
                e_i = 0.5 * (acc.e64[0] + acc.e64[1]);
                w_i = 0.5 * (acc.w64[0] + acc.w64[1]);
            }
        } else if (FP32) {
            long long *F = (long long *)v.F;
            FixedAcc fx;
            fx.zero();
            float f[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) f[a] = __fmaf_rn(s32, acc.f32[1][a], acc.f32[0][a]);
            // a NaN or a force beyond the fixed-point range (overlapping particles)
            // would be clamped by the conversion: report it instead
            if (!(fabsf(f[0]) < kFixedRange) || !(fabsf(f[1]) < kFixedRange) || !(fabsf(f[2]) < kFixedRange))
                atomicOr(&v.sc->flags, kFlagNonFinite);
            fx.add(f[0], f[1], f[2], fmaxf(fabsf(f[0]), fmaxf(fabsf(f[1]), fabsf(f[2]))));
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                qv[a] = fx.value(a);
                F[a * N + i] = qv[a];
            }
            if (ENERGY) {
                // the particle's energy and virial estimates in binary32, halved
                // exactly, then exactly in fixed point (scale 2^24): integer sums
                // over particles are exact and order-free, and need no FP64 pipe
                const float e = __fmul_rn(0.5f, __fmaf_rn(s32, acc.e32[1], acc.e32[0]));
                const float w = __fmul_rn(0.5f, __fmaf_rn(s32, acc.w32[1], acc.w32[0]));
                if (!(fabsf(e) < kEnergyRange) || !(fabsf(w) < kEnergyRange)) atomicOr(&v.sc->flags, kFlagNonFinite);
                eq = __float2ll_rn(__fmul_rn(e, 16777216.0f));
                wq = __float2ll_rn(__fmul_rn(w, 16777216.0f));
            }
        } else {
            double *F = (double *)v.F;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                f64[a] = acc.f64[0][a] + s64 * acc.f64[1][a];
                F[a * N + i] = f64[a];
            }
            e_i = 0.5 * (acc.e64[0] + s64 * acc.e64[1]);
            w_i = 0.5 * (acc.w64[0] + s64 * acc.w64[1]);
        }
    }
    // Total force and energy/virial partials.
    if (MODE == 2) {
        double x[2] = {e_i, w_i};
        group_sums<2>(x, v.partials, 3);
    } else if (FP32) {
        int lane = threadIdx.x & 31;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            long long s = warp_sum(qv[a]);
            if (lane == 0 && s != 0) atomicAdd(&v.rs[r].fsum_q[a], (unsigned long long)s);
        }
        if (ENERGY) { // a warp's slots belong to one replica (replicas start on whole tiles)
            const long long se = warp_sum(eq), sw = warp_sum(wq);
            if (lane == 0) {
                if (se != 0) atomicAdd(&v.rs[r].ew_q[0], (unsigned long long)se);
                if (sw != 0) atomicAdd(&v.rs[r].ew_q[1], (unsigned long long)sw);
            }
        }
    } else {
        double x[5] = {f64[0], f64[1], f64[2], e_i, w_i};
        group_sums<5>(x, v.partials, 0);
    }
}


// Launch k_force with the context's block size and its staging in dynamic shared
// memory (opting in to more than the default 48 KB where the largest block needs it).
// prepare = true: only set the shared-memory attribute (before a stream capture of
// this launch), launch nothing.
template <int MODE, bool FP32, bool ENERGY, int PMAX, bool EWALD>
cudaError_t launch_k_force(const View &v, int step_offset, cudaStream_t s, bool prepare = false)
{
    const int bd = v.force_threads;
    const size_t smem = (size_t)kMaskStage * bd * (sizeof(unsigned) + sizeof(unsigned short));
    if (smem > 40 * 1024) {
        // beyond the default limit together with the kernel's static shared memory:
        // a function attribute, set outside stream capture (the graphs of a step are
        // captured after a prepare call)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cs);
        if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone)
            e = cudaFuncSetAttribute(k_force<MODE, FP32, ENERGY, PMAX, EWALD>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (prepare) return cudaSuccess;
    k_force<MODE, FP32, ENERGY, PMAX, EWALD><<<ceil_div(v.N, bd), bd, smem, s>>>(v, step_offset);
    return cudaGetLastError();
}

template <int MODE, bool FP32, bool ENERGY, bool EWALD>
cudaError_t launch_force_p(const View &v, int step_offset, cudaStream_t s, bool prepare)
{
    if constexpr (MODE == 1) {
        return launch_k_force<MODE, FP32, ENERGY, 0, EWALD>(v, step_offset, s, prepare);
    } else {
        // every rank slot up to PMAX is resolved, so PMAX is p itself for the usual
        // batch sizes and a bound otherwise
        switch (v.p) {
        case 1: return launch_k_force<MODE, FP32, ENERGY, 1, EWALD>(v, step_offset, s, prepare);
        case 2: return launch_k_force<MODE, FP32, ENERGY, 2, EWALD>(v, step_offset, s, prepare);
        case 5: return launch_k_force<MODE, FP32, ENERGY, 5, EWALD>(v, step_offset, s, prepare);
        case 10: return launch_k_force<MODE, FP32, ENERGY, 10, EWALD>(v, step_offset, s, prepare);
        case 20: return launch_k_force<MODE, FP32, ENERGY, 20, EWALD>(v, step_offset, s, prepare);
        default:
            if (v.p <= 8) return launch_k_force<MODE, FP32, ENERGY, 8, EWALD>(v, step_offset, s, prepare);
            if (v.p <= 16) return launch_k_force<MODE, FP32, ENERGY, 16, EWALD>(v, step_offset, s, prepare);
            if (v.p <= 32) return launch_k_force<MODE, FP32, ENERGY, 32, EWALD>(v, step_offset, s, prepare);
            return launch_k_force<MODE, FP32, ENERGY, 0, EWALD>(v, step_offset, s, prepare);
        }
    }
}


// The force kernel for the context's mode, precision and batch size.
template <bool EWALD>
cudaError_t launch_force_dispatch(const View &v, int step_offset, bool energy, cudaStream_t s, bool prepare)
{
    bool fp32 = v.precision == RBL_FP32;
    if (v.full_list) {
        if (!fp32) return launch_force_p<1, false, true, EWALD>(v, step_offset, s, prepare);
        return energy ? launch_force_p<1, true, true, EWALD>(v, step_offset, s, prepare)
                      : launch_force_p<1, true, false, EWALD>(v, step_offset, s, prepare);
    }
    if (v.sampling) {
        if (!fp32) return launch_force_p<3, false, true, EWALD>(v, step_offset, s, prepare);
        return energy ? launch_force_p<3, true, true, EWALD>(v, step_offset, s, prepare)
                      : launch_force_p<3, true, false, EWALD>(v, step_offset, s, prepare);
    }
    if (!fp32) return launch_force_p<0, false, true, EWALD>(v, step_offset, s, prepare);
    return energy ? launch_force_p<0, true, true, EWALD>(v, step_offset, s, prepare)
                  : launch_force_p<0, true, false, EWALD>(v, step_offset, s, prepare);
}

// MODE 2 (exact energy and virial) in the context's precision.
template <bool EWALD>
cudaError_t launch_exact_dispatch(const View &v, cudaStream_t s)
{
    return v.precision == RBL_FP32 ? launch_k_force<2, true, true, 0, EWALD>(v, 0, s)
                                   : launch_k_force<2, false, true, 0, EWALD>(v, 0, s);
}

} // namespace

} // namespace rbl
