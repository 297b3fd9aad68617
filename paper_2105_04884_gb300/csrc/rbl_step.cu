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
// v + ck (F - F_cor).  k_integrate kicks with these same operations (ck = dt when
// it applies a pending closing half kick together with its own opening one); the
// velocities reported between steps are this with ck = dt/2.
template <bool FP32>
__device__ __forceinline__ double kick_v(const View &v, const RepScalars *rsc, int i, int tag, int a, double ck,
                                         double cks)
{
    const size_t N = (size_t)v.N;
    const double va = v.v[a * N + i];
    if (ck == 0.0) return va;
    if (FP32) {
        const long long q = ((const long long *)v.F)[a * N + i] - rsc->fcor_q[a] - (tag < rsc->fcor_r[a] ? 1 : 0);
        return fma(cks, __ll2double_rn(q), va); // exact: |q| < 2^53 (force range check)
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

// Observables launch, part 1: the kinetic sums of one tile (256 slots) per warp.
// Each lane sums its 8 slots in order (v^2 per axis, then the three added); the four
// per-lane sums (v^2, v_x, v_y, v_z) are
// then reduced over the warp by one fixed transposed shuffle tree (6 FP64 additions
// per lane instead of 20: the first level halves the values a lane carries, the
// second halves them again), after which lanes 8k hold the tile's sum of value k.
// ck: the half kick still pending at the end of a step call (the sums are of the
// kicked velocities).  Padding slots count as v = 0.  Each tile sum s is split
// exactly into floor(s) and the fraction s - floor(s) rounded to a multiple of 2^-40,
// both integers, and the replica's totals of those integers are accumulated by
// integer atomics: exact and order-free, so the result depends on the replica's
// tiles alone, never on the launch shape or on the other replicas of an ensemble.
// Part 2 (the block that finishes last) turns each replica's totals into one
// correctly rounded FP64 value and assembles rbl_obs.
constexpr int kObsBlock = 128;
constexpr double kTwo40 = 1099511627776.0;       // 2^40
constexpr double kKinRange = 4503599627370496.0; // 2^52: a tile sum beyond it is not split exactly

template <bool FP32>
__global__ void __launch_bounds__(kObsBlock) k_observables(View v, double ck, double cks, rbl_obs *out)
{
    constexpr int kWarps = kObsBlock / 32;
    __shared__ long long s_q[kWarps][8];
    __shared__ int s_rep[kWarps];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tile = blockIdx.x * kWarps + wid;
    if (tile < v.ntile) {
        const size_t base = (size_t)tile * kTile + lane;
        const int2 tl = v.tile[tile];
        const RepScalars *rsc = v.rs + tl.x;
        // per axis, so that no chain of dependent FP64 operations is longer than 8
        double q2[3] = {0, 0, 0}, x[4] = {0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < kTile / 32; ++k) {
            const size_t i = base + (size_t)k * 32;
            const bool live = (long long)i < (long long)tl.y;
            const int tag = live && ck != 0.0 ? v.tag[i] : 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double va = live ? kick_v<FP32>(v, rsc, (int)i, tag, a, ck, cks) : 0.0;
                q2[a] = fma(va, va, q2[a]);
                x[1 + a] += va;
            }
        }
        x[0] = (q2[0] + q2[1]) + q2[2];
        // level 16: lanes below 16 keep values 0, 1, the others 2, 3
        const bool u16 = (lane & 16) != 0;
        double a0 = u16 ? x[2] : x[0], a1 = u16 ? x[3] : x[1];
        const double o0 = u16 ? x[0] : x[2], o1 = u16 ? x[1] : x[3];
        a0 += __shfl_xor_sync(0xffffffffu, o0, 16);
        a1 += __shfl_xor_sync(0xffffffffu, o1, 16);
        // level 8: one value per lane, value 2 [lane & 16] + [lane & 8]
        const bool u8 = (lane & 8) != 0;
        double t = u8 ? a1 : a0;
        t += __shfl_xor_sync(0xffffffffu, u8 ? a0 : a1, 8);
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        if ((lane & 7) == 0) {
            const int k = lane >> 3;
            long long qi = 0, qf = 0;
            if (fabs(t) < kKinRange) {
                const double fl = floor(t);
                qi = (long long)fl;                      // exact: |fl| < 2^52
                qf = __double2ll_rn((t - fl) * kTwo40);  // t - fl exact, in [0, 1)
            } else {
                atomicOr(&v.sc->flags, kFlagNonFinite); // non-finite or absurd velocities
            }
            s_q[wid][2 * k] = qi;
            s_q[wid][2 * k + 1] = qf;
        }
        if (lane == 0) s_rep[wid] = tl.x;
    } else if (lane == 0) {
        s_rep[wid] = -1;
    }
    __syncthreads();
    // one atomic per value for each run of this block's warps in the same replica
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        unsigned long long *acc_k = v.kin_acc + (size_t)k * v.kin_stride;
        int rep = -1;
        long long acc = 0;
        for (int w = 0; w < kWarps; ++w) {
            if (s_rep[w] < 0) break;
            if (s_rep[w] != rep) {
                if (rep >= 0) atomicAdd(acc_k + rep, (unsigned long long)acc);
                rep = s_rep[w];
                acc = 0;
            }
            acc += s_q[w][k];
        }
        if (rep >= 0) atomicAdd(acc_k + rep, (unsigned long long)acc);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&v.sc->obs_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    // part 2: every block's totals are in; read and clear them
    __threadfence();
    for (int r = threadIdx.x; r < v.R; r += blockDim.x) {
        unsigned long long q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = atomicExch(v.kin_acc + (size_t)k * v.kin_stride + r, 0ull);
        double tot[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long qi = (long long)q[2 * k], qf = (long long)q[2 * k + 1];
            // exact integer part and exact fraction (< 1), one rounding in the add
            tot[k] = __dadd_rn((double)(qi + (qf >> 40)), __dmul_rn((double)(qf & ((1ll << 40) - 1)), 1.0 / kTwo40));
        }
        const RepScalars &s = v.rs[r];
        const Box &b = v.box[r];
        const double T_kin = __ddiv_rn(tot[0], b.n3);
        rbl_obs &o = out[r]; // written field by field (out may be mapped host memory)
        o.U_est = s.energy;
        o.W_est = s.virial;
        o.K = __dmul_rn(0.5, tot[0]);
        o.T_kin = T_kin;
        o.P = __dadd_rn(__dmul_rn(b.rho, T_kin), __ddiv_rn(s.virial, b.V3));
        o.U_tail = b.U_tail;
        o.P_tail = b.P_tail;
        for (int a = 0; a < 3; ++a) o.net_momentum[a] = tot[1 + a];
        o.step = (long long)v.sc->step;
        o.n_rebuild = s.n_rebuild;
        const double n = (double)b.N;
        o.Ns_mean = __ddiv_rn((double)s.ns_sum, n);
        o.Nc_mean = __ddiv_rn((double)s.nc_sum, n);
        o.Mc_mean = __ddiv_rn((double)s.m_sum, n);
        o.Ns_max = s.ns_max;
        o.Nc_max = s.nc_max;
    }
    if (threadIdx.x == 0) v.sc->obs_ticket = 0u;
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

cudaError_t launch_observables(const View &v, rbl_obs *out, double ck, cudaStream_t s)
{
    const int g = ceil_div(v.ntile, kObsBlock / 32);
    if (v.precision == RBL_FP32) k_observables<true><<<g, kObsBlock, 0, s>>>(v, ck, ck * kFixedInv, out);
    else k_observables<false><<<g, kObsBlock, 0, s>>>(v, ck, ck * kFixedInv, out);
    return cudaGetLastError();
}

} // namespace rbl
