// rbl_force.cu -- the RBL force (Sec. 2, Eqs. (3)-(4)), the classical full-list
// force, and the parity/observable kernels that share their pair rule.
//
// One thread per particle (cell order).  Core row: every entry with r < r_c is
// summed.  Shell row: a Floyd p-subset of positions is drawn from Philox stream 0 of
// (seed, step, tag) -- or the whole row when N_s <= p -- and every drawn entry with
// r_c <= r < r_s contributes s f_ij, s = N_s / p.
//
// FP32 path: pair arithmetic in binary32, each pair's force (times s) converted
// exactly to fixed point at scale 2^24 and summed in integers, so the sum does not
// depend on the order or on the thread mapping; the total force is accumulated
// with 64-bit integer atomics (exact).  FP64 path: FP64 pair arithmetic from the
// FP64 positions, per-block partial sums reduced in a fixed order.
#include "rbl_internal.cuh"

namespace rbl {

namespace {

struct Pair64 {
    double f[3];
    double u, w;
};

// FP64 pair force from FP64 positions (minimum image by rounding d/L).
__device__ __forceinline__ void pair64(const View &v, int i, int j, Pair64 &out)
{
    size_t N = (size_t)v.N;
    double r2 = 0.0;
    double d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double t = v.x[a * N + i] - v.x[a * N + j];
        t -= v.L[a] * rint(t / v.L[a]);
        d[a] = t;
    }
    r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double inv = 1.0 / r2;
    double r6 = inv * inv * inv;
    double vir = 24.0 * (2.0 * r6 * r6 - r6);
    double coef = vir * inv;
    out.f[0] = coef * d[0];
    out.f[1] = coef * d[1];
    out.f[2] = coef * d[2];
    out.u = 4.0 * (r6 * r6 - r6);
    out.w = vir;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Deterministic block sum (fixed tree) of NV doubles per thread into out[0..NV).
template <int NV>
__device__ __forceinline__ void block_sum_d(double (&x)[NV], double *out)
{
    __shared__ double sh[NV][kBlock / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(x[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += sh[threadIdx.x][w];
        out[threadIdx.x] = s;
    }
}

// MODE 0: RBL (core + sampled shell); MODE 1: full list (rows in the shell arrays).
template <int MODE, bool FP32, bool ENERGY>
__global__ void __launch_bounds__(kBlock) k_force(View v, int step_offset)
{
    const unsigned long long step = v.sc->step + (unsigned long long)step_offset;
    int i = blockIdx.x * kBlock + threadIdx.x;
    bool active = i < v.N;
    long long q[3] = {0, 0, 0};
    double f64[3] = {0.0, 0.0, 0.0};
    double e_i = 0.0, w_i = 0.0;
    if (active) {
        int4 pi = v.pos[i];
        FixedAcc acc;
        acc.zero();
        float e_c = 0.f, w_c = 0.f, e_s = 0.f, w_s = 0.f;
        double e_c64 = 0.0, w_c64 = 0.0, e_s64 = 0.0, w_s64 = 0.0;
        double fc[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
        if (MODE == 0) {
            int nc = min(v.n_core[i], v.cap_c);
            const int *crow = v.core + (size_t)i * v.cap_c;
            for (int k = 0; k < nc; ++k) {
                int j = crow[k];
                PairGeom g = pair_geom(pi, v.pos[j], v.h);
                bool in = g.r2 < v.t_rc2;
                if (FP32) {
                    float u, w;
                    float coef = lj_coef(g.r2, &u, &w);
                    coef = in ? coef : 0.f;
                    acc.add(__fmul_rn(coef, g.dx), __fmul_rn(coef, g.dy), __fmul_rn(coef, g.dz));
                    if (ENERGY && in) {
                        e_c += u;
                        w_c += w;
                    }
                } else if (in) {
                    Pair64 pr;
                    pair64(v, i, j, pr);
#pragma unroll
                    for (int a = 0; a < 3; ++a) fc[a] += pr.f[a];
                    e_c64 += pr.u;
                    w_c64 += pr.w;
                }
            }
        }
        int ns = min(v.n_shell[i], v.cap_s);
        const int *srow = v.shell + (size_t)i * v.cap_s;
        int S[kMaxP];
        int nb;
        float s32 = 1.0f;
        double s64 = 1.0;
        if (MODE == 0) {
            nb = floyd_positions(v.seed, step, pi.w, ns, v.p, S, &v.sc->flags);
            if (ns > v.p) {
                s32 = __fdiv_rn((float)ns, (float)v.p);
                s64 = (double)ns / (double)v.p;
            }
        } else {
            nb = ns;
        }
        for (int q_ = 0; q_ < nb; ++q_) {
            int j = srow[MODE == 0 ? S[q_] : q_];
            PairGeom g = pair_geom(pi, v.pos[j], v.h);
            bool in = MODE == 0 ? (g.r2 >= v.t_rc2 && g.r2 < v.t_rs2) : (g.r2 < v.t_rs2);
            if (FP32) {
                float u, w;
                float coef = lj_coef(g.r2, &u, &w);
                coef = in ? coef : 0.f;
                acc.add(__fmul_rn(__fmul_rn(coef, g.dx), s32), __fmul_rn(__fmul_rn(coef, g.dy), s32),
                        __fmul_rn(__fmul_rn(coef, g.dz), s32));
                if (ENERGY && in) {
                    e_s += u;
                    w_s += w;
                }
            } else if (in) {
                Pair64 pr;
                pair64(v, i, j, pr);
#pragma unroll
                for (int a = 0; a < 3; ++a) fs[a] += pr.f[a];
                e_s64 += pr.u;
                w_s64 += pr.w;
            }
        }
        size_t N = (size_t)v.N;
        if (FP32) {
            long long *F = (long long *)v.F;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                q[a] = acc.value(a);
                F[a * N + i] = q[a];
            }
            if (ENERGY) {
                e_i = 0.5 * ((double)e_c + (double)s32 * (double)e_s);
                w_i = 0.5 * ((double)w_c + (double)s32 * (double)w_s);
            }
        } else {
            double *F = (double *)v.F;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                f64[a] = fc[a] + s64 * fs[a];
                F[a * N + i] = f64[a];
            }
            e_i = 0.5 * (e_c64 + s64 * e_s64);
            w_i = 0.5 * (w_c64 + s64 * w_s64);
        }
    }
    // Total force and energy/virial partials.
    if (FP32) {
        int lane = threadIdx.x & 31;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            long long s = warp_sum(q[a]);
            if (lane == 0 && s != 0) atomicAdd(&v.sc->fsum_q[a], (unsigned long long)s);
        }
        if (ENERGY) {
            double x[2] = {e_i, w_i};
            block_sum_d<2>(x, v.partials + (size_t)blockIdx.x * 8 + 3);
        }
    } else {
        double x[5] = {f64[0], f64[1], f64[2], e_i, w_i};
        block_sum_d<5>(x, v.partials + (size_t)blockIdx.x * 8);
    }
}

// Reduce the block partials in a fixed order; form the mean force F_cor
// (Appendix A) and reset the integer accumulator for the next evaluation.
__global__ void __launch_bounds__(1024) k_force_finish(View v, int nblk, int fp32, int energy, int subtract,
                                                       int advance)
{
    __shared__ double sh[5][32];
    double acc[5] = {0, 0, 0, 0, 0};
    if (fp32 && !energy) nblk = 0; // only the integer total is needed
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += v.partials[(size_t)b * 8 + k];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double s = warp_sum(acc[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 5; ++k) tot[k] += sh[k][w];
        DevScalars *sc = v.sc;
        for (int a = 0; a < 3; ++a) {
            double m;
            if (fp32) {
                long long qs = (long long)sc->fsum_q[a];
                m = (double)qs * kFixedInv / (double)v.N;
                sc->fsum_q[a] = 0ull;
            } else {
                m = tot[a] / (double)v.N;
            }
            sc->fcor[a] = subtract ? m : 0.0;
        }
        if (energy) {
            sc->energy = tot[3];
            sc->virial = tot[4];
        }
        sc->step += (unsigned long long)advance;
    }
}

// Mean-subtracted force, scattered to tag order as AoS doubles.
__global__ void k_store_forces(View v, double *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    size_t N = (size_t)v.N;
    int t = v.tag[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double f = v.precision == RBL_FP32 ? (double)((const long long *)v.F)[a * N + i] * kFixedInv
                                           : ((const double *)v.F)[a * N + i];
        out[(size_t)t * 3 + a] = f - v.sc->fcor[a];
    }
}

// Batch positions B(i) for `step` (parity hook): out_pos[i][p] (row positions,
// draw order), out_n[i].
__global__ void k_batch(View v, unsigned long long step, int *out_pos, int *out_n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    int ns = min(v.n_shell[i], v.cap_s);
    int S[kMaxP];
    int nb = floyd_positions(v.seed, step, v.pos[i].w, ns, v.p, S, &v.sc->flags);
    for (int q = 0; q < nb; ++q) out_pos[(size_t)i * v.p + q] = S[q];
    out_n[i] = nb;
}

// g(r) counts: every pair once per ordered (i, j), classified like the force.
__global__ void k_rdf(View v, float dr, int nbins, unsigned long long *hist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    int4 pi = v.pos[i];
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 0 && v.full_list) continue;
        const int *row = pass == 0 ? v.core + (size_t)i * v.cap_c : v.shell + (size_t)i * v.cap_s;
        int n = pass == 0 ? min(v.n_core[i], v.cap_c) : min(v.n_shell[i], v.cap_s);
        for (int k = 0; k < n; ++k) {
            PairGeom g = pair_geom(pi, v.pos[row[k]], v.h);
            bool in;
            if (v.full_list) in = g.r2 < v.t_rs2;
            else in = pass == 0 ? g.r2 < v.t_rc2 : (g.r2 >= v.t_rc2 && g.r2 < v.t_rs2);
            if (!in) continue;
            float qf = __fdiv_rn(__fsqrt_rn(g.r2), dr);
            if (qf < (float)nbins) atomicAdd(&hist[(int)qf], 1ull);
        }
    }
}

} // namespace

cudaError_t launch_force_kernel(const View &v, int step_offset, bool energy, cudaStream_t s)
{
    int g = ceil_div(v.N, kBlock);
    bool fp32 = v.precision == RBL_FP32;
    if (v.full_list) {
        if (fp32) {
            if (energy) k_force<1, true, true><<<g, kBlock, 0, s>>>(v, step_offset);
            else k_force<1, true, false><<<g, kBlock, 0, s>>>(v, step_offset);
        } else {
            k_force<1, false, true><<<g, kBlock, 0, s>>>(v, step_offset);
        }
    } else {
        if (fp32) {
            if (energy) k_force<0, true, true><<<g, kBlock, 0, s>>>(v, step_offset);
            else k_force<0, true, false><<<g, kBlock, 0, s>>>(v, step_offset);
        } else {
            k_force<0, false, true><<<g, kBlock, 0, s>>>(v, step_offset);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_force_finish(const View &v, int advance, bool energy, cudaStream_t s)
{
    int g = ceil_div(v.N, kBlock);
    bool fp32 = v.precision == RBL_FP32;
    k_force_finish<<<1, 1024, 0, s>>>(v, g, fp32 ? 1 : 0, (energy || !fp32) ? 1 : 0, v.subtract, advance);
    return cudaGetLastError();
}

cudaError_t launch_forces(const View &v, int step_offset, int advance, bool energy, cudaStream_t s)
{
    cudaError_t e = launch_force_kernel(v, step_offset, energy, s);
    if (e == cudaSuccess) e = launch_force_finish(v, advance, energy, s);
    return e;
}

cudaError_t launch_store_forces(const View &v, double *F, cudaStream_t s)
{
    k_store_forces<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, F);
    return cudaGetLastError();
}

cudaError_t launch_batch(const View &v, unsigned long long step, int *out_pos, int *out_n, cudaStream_t s)
{
    k_batch<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, step, out_pos, out_n);
    return cudaGetLastError();
}

cudaError_t launch_rdf(const View &v, float dr, int nbins, unsigned long long *hist, cudaStream_t s)
{
    k_rdf<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, dr, nbins, hist);
    return cudaGetLastError();
}

} // namespace rbl
