// rbl_step.cu -- state I/O, the fused kick/drift/thermostat kernel and the
// kinetic reductions (Algorithm 1; Sec. 2, Eq. (2); Sec. 3).
//
// Time stepping is velocity-Verlet for the underdamped Langevin equation in the
// BAOAB splitting: B: v += dt/2 F~, A: x += dt/2 v, O: v = c1 v + c2 xi,
// A: x += dt/2 v, force, B.  The closing B of one step and the opening B of the
// next use the same force, so inside a multi-step call they are one kick of dt.
// gamma = 0 gives plain velocity-Verlet (single drift of dt).  Positions, velocities
// and the kicks are FP64; the thermostat noise xi is drawn in binary32 (Box-Muller
// on Philox stream 1) and widened.  The kernel also refreshes the 32-bit
// fixed-point image used by the pair rule and raises the rebuild flag when a
// particle has moved more than skin/2 since the last build.
#include "rbl_internal.cuh"

namespace rbl {

namespace {

// Load packed AoS tag-ordered x (and v) into the SoA arrays (identity order within
// each replica: slot first + t holds tag t), wrap x into [0, L), refresh the
// fixed-point image, and flag non-finite input.  Padding slots are cleared.
__global__ void k_load(View v, const double *x, const double *vel)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    size_t N = (size_t)v.N;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) {
#pragma unroll
        for (int a = 0; a < 3; ++a) v.x[a * N + i] = v.v[a * N + i] = 0.0;
        v.tag[i] = 0;
        v.pos[i] = v.ubuild[i] = make_int4(0, 0, 0, 0);
        if (v.q) {
            v.q[i] = 0.0;
            v.q32[i] = 0.f;
        }
        return;
    }
    const Box &b = v.box[r];
    const int t = i - b.first;
    const size_t row = (size_t)b.in0 + (size_t)t;
    unsigned u[3];
    bool bad = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double xa = x[row * 3 + a];
        double va = vel ? vel[row * 3 + a] : 0.0;
        bad |= !isfinite(xa) || !isfinite(va);
        if (!isfinite(xa)) xa = 0.0;
        xa = xa - b.L[a] * floor(xa / b.L[a]);
        if (xa >= b.L[a]) xa -= b.L[a];
        if (xa < 0.0) xa = 0.0;
        v.x[a * N + i] = xa;
        v.v[a * N + i] = va;
        u[a] = quantize(xa, b.inv[a]);
    }
    v.tag[i] = t;
    v.pos[i] = make_int4((int)u[0], (int)u[1], (int)u[2], t);
    v.ubuild[i] = v.pos[i];
    if (v.q) {
        v.q[i] = v.q_in[i];
        v.q32[i] = __double2float_rn(v.q_in[i]);
    }
    if (bad) atomicOr(&v.sc->flags, kFlagNonFinite);
}

// Charges from packed tag-ordered input: into load order (slot first + t for tag
// t, zero on padding slots) and, through each slot's tag, into the current order.
__global__ void k_set_charges(View v, const double *q)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) {
        v.q_in[i] = v.q[i] = 0.0;
        v.q32[i] = 0.f;
        return;
    }
    const Box &b = v.box[r];
    v.q_in[i] = q[(size_t)b.in0 + (size_t)(i - b.first)];
    const double qi = q[(size_t)b.in0 + (size_t)v.tag[i]];
    v.q[i] = qi;
    v.q32[i] = __double2float_rn(qi);
}

// Velocity component a of slot i after a kick of ck by the corrected force (ck 0:
// no kick).  FP32 path: the corrected force is the integer q_i - m - [tag < r] (the
// net force removed exactly, see k_force_finish), converted exactly and applied with
// one fused multiply-add, v + (ck 2^-24) (q_i - m - [tag < r]); FP64 path:
// v + ck (F - F_cor).  k_integrate kicks with these same operations, so a kick
// computed here for output equals the one the next step applies.
template <bool FP32>
__device__ __forceinline__ double kick_v(const View &v, const RepScalars *rsc, int i, int tag, int a, double ck,
                                         double cks)
{
    const size_t N = (size_t)v.N;
    const double va = v.v[a * N + i];
    if (ck == 0.0) return va;
    if (FP32) {
        const long long q = ((const long long *)v.F)[a * N + i] - rsc->fcor_q[a] - (tag < rsc->fcor_r[a] ? 1 : 0);
        return fma(cks, i64_to_double(q), va);
    }
    return fma(ck, ((const double *)v.F)[a * N + i] - rsc->fcor[a], va);
}

// SoA cell-ordered state -> packed AoS tag-ordered output; ck: the half kick still
// pending at the end of a step call, applied to the velocities written (the state
// keeps them unkicked).
template <bool FP32>
__global__ void k_store(View v, double *x, double *vel, double ck, double cks)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    size_t N = (size_t)v.N;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    const int tag = v.tag[i];
    size_t t = (size_t)v.box[r].in0 + (size_t)tag;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (x) x[t * 3 + a] = v.x[a * N + i];
        if (vel) vel[t * 3 + a] = kick_v<FP32>(v, v.rs + r, i, tag, a, ck, cks);
    }
}

// Checkpoint I/O, tag order packed over replicas: the images of the last build,
// out of cell order (k_store_images) and into load order, slot first + t for tag t
// (k_load_images, after k_load).
__global__ void k_store_images(View v, unsigned *img)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    const size_t t = (size_t)v.box[r].in0 + (size_t)v.tag[i];
    const int4 u = v.ubuild[i];
    img[t * 3 + 0] = (unsigned)u.x;
    img[t * 3 + 1] = (unsigned)u.y;
    img[t * 3 + 2] = (unsigned)u.z;
}

__global__ void k_load_images(View v, const unsigned *img)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    const Box &b = v.box[r];
    const int t = i - b.first;
    const size_t row = (size_t)b.in0 + (size_t)t;
    v.ubuild[i] = make_int4((int)img[row * 3 + 0], (int)img[row * 3 + 1], (int)img[row * 3 + 2], t);
}

// The current fixed-point images from the FP64 positions (slot order as it stands).
__global__ void k_requantize(View v)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    const Box &b = v.box[r];
    const size_t N = (size_t)v.N;
    v.pos[i] = make_int4((int)quantize(v.x[i], b.inv[0]), (int)quantize(v.x[N + i], b.inv[1]),
                         (int)quantize(v.x[2 * N + i], b.inv[2]), v.tag[i]);
}

// ck: kick coefficient (dt/2 or dt); cks = ck 2^-24, the kick per fixed-point unit
// of force.  DRIFT = false: kick only (closing half-kick).
//
// FP32 path: the corrected force of particle i is the integer q_i - m - [tag < r]
// (the net force removed exactly, see k_force_finish), converted exactly and
// applied with one fused multiply-add: v += cks (q_i - m - [tag < r]).
template <bool FP32, bool LANGEVIN, bool DRIFT>
__global__ void __launch_bounds__(kBlock) k_integrate(View v, double ck, double cks)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    const Box &b = v.box[r];
    size_t N = (size_t)v.N;
    const RepScalars *rsc = v.rs + r;
    const int tag = v.tag[i];
    double vv[3], xx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) vv[a] = kick_v<FP32>(v, rsc, i, tag, a, ck, cks);
    if constexpr (!DRIFT) {
#pragma unroll
        for (int a = 0; a < 3; ++a) v.v[a * N + i] = vv[a];
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) xx[a] = v.x[a * N + i];
        if (LANGEVIN) {
            const double half = 0.5 * v.dt;
#pragma unroll
            for (int a = 0; a < 3; ++a) xx[a] = fma(half, vv[a], xx[a]);
            // O-step noise: Box-Muller of a_k = ((w_k >> 9) + 1/2) 2^-23, stream 1.
            WordStream ws;
            ws.init(b.seed, v.sc->step, (uint32_t)tag, 1u);
            float av[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                av[k] = __fmul_rn(__fadd_rn((float)(ws.next() >> 9), 0.5f), 1.1920928955078125e-7f);
            float r0 = sqrtf(-2.0f * logf(av[0]));
            float r1 = sqrtf(-2.0f * logf(av[2]));
            float s1, c1v;
            sincospif(2.0f * av[1], &s1, &c1v);
            float c3 = cospif(2.0f * av[3]);
            float xi[3] = {r0 * c1v, r0 * s1, r1 * c3};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double noise = f32_to_double(b.c2f * xi[a]);
                vv[a] = fma(v.c1, vv[a], noise);
                xx[a] = fma(half, vv[a], xx[a]);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) xx[a] = fma(v.dt, vv[a], xx[a]);
        }
        unsigned u[3];
        bool bad = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double xa = wrap(xx[a], b.L[a]);
            // non-finite, or still outside the box: a step of more than a box length
            bad |= !finite_bits(xa) || !finite_bits(vv[a]) || !in_box_bits(xa, b.L[a]);
            v.x[a * N + i] = xa;
            v.v[a * N + i] = vv[a];
            u[a] = quantize(xa, b.inv[a]);
        }
        int4 np = make_int4((int)u[0], (int)u[1], (int)u[2], tag);
        v.pos[i] = np;
        PairGeom g = pair_geom(np, v.ubuild[i], b.h);
        if (g.r2 > v.t_disp) {
            v.rs[r].rebuild = 1;
            v.sc->rebuild = 1;
        }
        if (bad) atomicOr(&v.sc->flags, kFlagNonFinite);
    }
}

template <typename T>
__device__ __forceinline__ T wsum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// sum v^2 and sum v per tile (256 slots): one warp per tile, each lane summing its
// 8 slots in order before one fixed shuffle tree, so the FP64 tree is paid once
// per 256 particles; per-tile partials in staging, reduced per replica in a fixed
// order by k_kinetic_finish.  Padding slots count as v = 0.  ck: the half kick still
// pending at the end of a step call (the sums are of the kicked velocities).
template <bool FP32>
__global__ void __launch_bounds__(32) k_kinetic(View v, double ck, double cks)
{
    const size_t N = (size_t)v.N;
    const size_t base = (size_t)blockIdx.x * kTile + threadIdx.x;
    const int2 tl = v.tile[blockIdx.x];
    const RepScalars *rsc = v.rs + tl.x;
    double x[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < kTile / 32; ++k) {
        const size_t i = base + (size_t)k * 32;
        const bool live = (long long)i < (long long)tl.y;
        const int tag = live && ck != 0.0 ? v.tag[i] : 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double va = live ? kick_v<FP32>(v, rsc, (int)i, tag, a, ck, cks) : 0.0;
            x[0] = fma(va, va, x[0]);
            x[1 + a] += va;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = wsum(x[k]);
    if (threadIdx.x < 4) {
        const double out = threadIdx.x == 0 ? x[0] : threadIdx.x == 1 ? x[1] : threadIdx.x == 2 ? x[2] : x[3];
        v.staging[(size_t)blockIdx.x * 4 + threadIdx.x] = out;
    }
}

__global__ void __launch_bounds__(kBlock) k_kinetic_finish(View v)
{
    __shared__ double sh[4][kBlock / 32];
    const Box &bx = v.box[blockIdx.x];
    const int t0 = bx.first >> kTileShift, nt = bx.slots >> kTileShift;
    double acc[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nt; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += v.staging[(size_t)(t0 + b) * 4 + k];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double s = wsum(acc[k]);
        if (lane == 0) sh[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[4] = {0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int k = 0; k < 4; ++k) tot[k] += sh[k][w];
        RepScalars &rsc = v.rs[blockIdx.x];
        rsc.ksum = tot[0];
        for (int a = 0; a < 3; ++a) rsc.psum[a] = tot[1 + a];
    }
}

// Density profile along one axis (Sec. 3 observables): particle counts in nbins
// slabs of equal width, bin = floor(u_a nbins / 2^32) from the fixed-point image
// (exact, and the same rule that assigns cells).  Shared-memory histogram per
// block (a block lies in one replica), then one global add per bin; hist[R][nbins].
__global__ void k_profile(View v, int axis, int nbins, unsigned long long *hist)
{
    extern __shared__ unsigned s_hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) s_hist[b] = 0u;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool live = false;
    const int r = i < v.N ? slot_replica(v, i, live) : v.tile[(v.N - 1) >> kTileShift].x;
    if (live) {
        const int4 p = v.pos[i];
        const unsigned u = axis == 0 ? (unsigned)p.x : (axis == 1 ? (unsigned)p.y : (unsigned)p.z);
        atomicAdd(&s_hist[(int)(((unsigned long long)u * (unsigned)nbins) >> 32)], 1u);
    }
    __syncthreads();
    unsigned long long *hr = hist + (size_t)r * nbins;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&hr[b], (unsigned long long)s_hist[b]);
}

// Replica tables of a context of one system, written on the device so that a
// caller that may not allocate host memory can set them up (replica 0 owns every
// tile and cell).
__global__ void k_init_single(View v, Box b)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) *const_cast<Box *>(v.box) = b;
    if (k < v.ntile) const_cast<int2 *>(v.tile)[k] = make_int2(0, b.first + b.N);
    if (k < v.ncell) const_cast<int *>(v.cell_rep)[k] = 0;
}

} // namespace

cudaError_t launch_profile(const View &v, int axis, int nbins, unsigned long long *hist, cudaStream_t s)
{
    k_profile<<<ceil_div(v.N, kBlock), kBlock, (size_t)nbins * 4, s>>>(v, axis, nbins, hist);
    return cudaGetLastError();
}

cudaError_t launch_init_single(const View &v, const Box &b, cudaStream_t s)
{
    int n = v.ntile > v.ncell ? v.ntile : v.ncell;
    k_init_single<<<ceil_div(n, kBlock), kBlock, 0, s>>>(v, b);
    return cudaGetLastError();
}

cudaError_t launch_load_state(const View &v, const double *x, const double *vel, cudaStream_t s)
{
    k_load<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, x, vel);
    return cudaGetLastError();
}

cudaError_t launch_set_charges(const View &v, const double *q_packed, cudaStream_t s)
{
    k_set_charges<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, q_packed);
    return cudaGetLastError();
}

cudaError_t launch_store_images(const View &v, unsigned *img, cudaStream_t s)
{
    k_store_images<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, img);
    return cudaGetLastError();
}

cudaError_t launch_load_images(const View &v, const unsigned *img, cudaStream_t s)
{
    k_load_images<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, img);
    return cudaGetLastError();
}

cudaError_t launch_requantize(const View &v, cudaStream_t s)
{
    k_requantize<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_store_state(const View &v, double *x, double *vel, cudaStream_t s, double ck)
{
    if (v.precision == RBL_FP32) k_store<true><<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, x, vel, ck, ck * kFixedInv);
    else k_store<false><<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, x, vel, ck, ck * kFixedInv);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const View &v, double ck, bool drift, cudaStream_t s)
{
    int g = ceil_div(v.N, kBlock);
    bool fp32 = v.precision == RBL_FP32;
    bool lang = v.gamma > 0.0;
    const double cks = ck * kFixedInv;
    if (!drift) {
        if (fp32) k_integrate<true, false, false><<<g, kBlock, 0, s>>>(v, ck, cks);
        else k_integrate<false, false, false><<<g, kBlock, 0, s>>>(v, ck, cks);
    } else if (fp32) {
        if (lang) k_integrate<true, true, true><<<g, kBlock, 0, s>>>(v, ck, cks);
        else k_integrate<true, false, true><<<g, kBlock, 0, s>>>(v, ck, cks);
    } else {
        if (lang) k_integrate<false, true, true><<<g, kBlock, 0, s>>>(v, ck, cks);
        else k_integrate<false, false, true><<<g, kBlock, 0, s>>>(v, ck, cks);
    }
    return cudaGetLastError();
}

// rbl_obs of every replica from its scalars (kinetic sums, energy and virial of the
// last force evaluation, list statistics): out[R], for rbl_observables and its
// asynchronous form alike.  Explicitly rounded operations, no contraction.
__global__ void k_obs(View v, rbl_obs *out, double rs)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= v.R) return;
    const double pi = 3.14159265358979323846;
    const RepScalars &s = v.rs[r];
    const Box &b = v.box[r];
    const double n = (double)b.N;
    const double V = __dmul_rn(__dmul_rn(b.L[0], b.L[1]), b.L[2]);
    const double rho = __ddiv_rn(n, V);
    const double i3 = __ddiv_rn(1.0, __dmul_rn(__dmul_rn(rs, rs), rs));
    const double i9 = __dmul_rn(__dmul_rn(i3, i3), i3);
    rbl_obs o;
    o.U_est = s.energy;
    o.W_est = s.virial;
    o.K = __dmul_rn(0.5, s.ksum);
    o.T_kin = __ddiv_rn(s.ksum, __dmul_rn(3.0, n));
    o.P = __dadd_rn(__dmul_rn(rho, o.T_kin), __ddiv_rn(s.virial, __dmul_rn(3.0, V)));
    // per-particle energy and pressure tails of the truncated LJ fluid (Sec. 3)
    o.U_tail = __dmul_rn(__dmul_rn(__dmul_rn(__ddiv_rn(8.0, 3.0), pi), rho), __dsub_rn(__ddiv_rn(i9, 3.0), i3));
    o.P_tail = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(__ddiv_rn(16.0, 3.0), pi), rho), rho),
                         __dsub_rn(__ddiv_rn(__dmul_rn(2.0, i9), 3.0), i3));
    for (int a = 0; a < 3; ++a) o.net_momentum[a] = s.psum[a];
    o.step = (long long)v.sc->step;
    o.n_rebuild = s.n_rebuild;
    o.Ns_mean = __ddiv_rn((double)s.ns_sum, n);
    o.Nc_mean = __ddiv_rn((double)s.nc_sum, n);
    o.Mc_mean = __ddiv_rn((double)s.m_sum, n);
    o.Ns_max = s.ns_max;
    o.Nc_max = s.nc_max;
    out[r] = o;
}

cudaError_t launch_obs(const View &v, rbl_obs *out, double rs, cudaStream_t s)
{
    k_obs<<<ceil_div(v.R, 128), 128, 0, s>>>(v, out, rs);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(const View &v, cudaStream_t s, double ck)
{
    if (v.precision == RBL_FP32) k_kinetic<true><<<v.ntile, 32, 0, s>>>(v, ck, ck * kFixedInv);
    else k_kinetic<false><<<v.ntile, 32, 0, s>>>(v, ck, ck * kFixedInv);
    k_kinetic_finish<<<v.R, kBlock, 0, s>>>(v);
    return cudaGetLastError();
}

} // namespace rbl
