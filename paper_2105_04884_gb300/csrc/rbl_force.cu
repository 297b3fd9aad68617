// rbl_force.cu -- the RBL force (Sec. 2, Eqs. (3)-(4)) and the classical full-list
// force with the LJ pair (the kernel itself is in rbl_force_kernel.cuh), the
// reductions that follow them, and the parity/observable kernels that share their
// pair rule.
#include "rbl_force_kernel.cuh"

namespace rbl {

namespace {

// Second stage of the per-replica sums (FP64 forces, energies): block (c, r) adds
// the partials of chunk c of replica r -- its 64-thread groups c*256 .. c*256+255 --
// in a fixed tree, one group per thread, so the per-replica reduction reads one
// entry per chunk instead of one per group and the work is spread over the GPU.
// The tree depends on neither the force kernel's block size nor the ensemble.
__global__ void __launch_bounds__(kChunkGroups) k_force_chunks(View v)
{
    const int c = blockIdx.x, r = blockIdx.y;
    const Box &b = v.box[r];
    const int g0 = b.first / kMinBlock, ng = b.slots / kMinBlock;
    if (c * kChunkGroups >= ng) return; // block-uniform: past this replica's groups
    const int g = c * kChunkGroups + (int)threadIdx.x;
    double x[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) x[q] = g < ng ? v.partials[(size_t)(g0 + g) * 8 + q] : 0.0;
    __shared__ double sh[5][kChunkGroups / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double s = warp_sum(x[q]);
        if (lane == 0) sh[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int w = 0; w < kChunkGroups / 32; ++w) t += sh[threadIdx.x][w];
        v.partials2[((size_t)r * v.pchunks + c) * 8 + threadIdx.x] = t;
    }
}

// One block per replica: reduce its chunks' sums (k_force_chunks) in a fixed order,
// form its mean force F_cor (Appendix A) and reset its integer accumulator for the
// next evaluation.  The FP32 path without energies reads no partials (its net force
// is the exact integer sum).  exact = 1: store the unsampled energy and virial only
// (MODE 2 partials).
__global__ void __launch_bounds__(kBlock) k_force_finish(View v, int fp32, int energy, int subtract, int advance,
                                                         int exact)
{
    __shared__ double sh[5][kBlock / 32];
    const int r = blockIdx.x;
    const Box &b = v.box[r];
    const int ng = b.slots / kMinBlock;
    // the FP32 path's sums are exact integers in rs (forces, energies): no partials
    const int nb = (fp32 && !exact) ? 0 : (ng + kChunkGroups - 1) / kChunkGroups;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) acc[q] += v.partials2[((size_t)r * v.pchunks + k) * 8 + q];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        double s = warp_sum(acc[q]);
        if (lane == 0) sh[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            for (int q = 0; q < 5; ++q) tot[q] += sh[q][w];
        RepScalars &rsc = v.rs[r];
        if (exact) {
            rsc.u_exact = tot[3];
            rsc.w_exact = tot[4];
            return;
        }
        for (int a = 0; a < 3; ++a) {
            double m;
            if (fp32) {
                // the net force Q, exact in fixed point, is removed exactly: Q = N m + rem
                // with 0 <= rem < N, and the rem particles of lowest tag take one unit
                // more, so the corrected forces sum to zero (momentum is conserved)
                const long long Q = subtract ? (long long)rsc.fsum_q[a] : 0ll;
                long long mq = Q / b.N, rq = Q - mq * b.N;
                if (rq < 0) {
                    mq -= 1;
                    rq += b.N;
                }
                rsc.fcor_q[a] = mq;
                rsc.fcor_r[a] = rq;
                m = (double)Q * kFixedInv / (double)b.N;
                rsc.fsum_q[a] = 0ull;
            } else {
                m = subtract ? tot[a] / (double)b.N : 0.0;
            }
            rsc.fcor[a] = m;
        }
        if (energy) {
            if (fp32) {
                const double sc = 1.0 / 16777216.0;
                rsc.energy = (double)(long long)rsc.ew_q[0] * sc;
                rsc.virial = (double)(long long)rsc.ew_q[1] * sc;
                rsc.ew_q[0] = rsc.ew_q[1] = 0ull;
            } else {
                rsc.energy = tot[3];
                rsc.virial = tot[4];
            }
        }
        if (r == 0) v.sc->step += (unsigned long long)advance;
    }
}

// Mean-subtracted force, scattered to tag order as AoS doubles.
__global__ void k_store_forces(View v, double *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    size_t N = (size_t)v.N;
    const int tag = v.tag[i];
    size_t t = (size_t)v.box[r].in0 + (size_t)tag;
    const RepScalars &rsc = v.rs[r];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (v.precision == RBL_FP32) {
            const long long q = ((const long long *)v.F)[a * N + i] - rsc.fcor_q[a] - (tag < rsc.fcor_r[a] ? 1 : 0);
            out[t * 3 + a] = (double)q * kFixedInv;
        } else {
            out[t * 3 + a] = ((const double *)v.F)[a * N + i] - rsc.fcor[a];
        }
    }
}

// Batch B(i) for `step` (parity hook): out_j[i][p] = neighbour indices in ascending
// row position, out_n[i] = their number.
__global__ void k_batch(View v, unsigned long long step, int *out_j, int *out_n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) {
        out_n[i] = 0;
        return;
    }
    const size_t N = (size_t)v.N;
    const int4 pi = v.pos[i];
    const int ns = v.n_shell[i];
    int S[kMaxP];
    const int nb = floyd_positions(v.box[r].seed, step, pi.w, ns, v.p, S, &v.sc->flags);
    sort_small(S, nb);
    SegCursor cur;
    const int4 *tab = v.seg_tab + (size_t)v.hcell[i] * v.S;
    cur.init(tab);
    if (v.sampling) {
        const int self = pool_self_position(v.box[r], tab, i);
        for (int q = 0; q < nb; ++q) out_j[(size_t)i * v.p + q] = cur.index_of(S[q] + (S[q] >= self ? 1 : 0));
        out_n[i] = nb;
        return;
    }
    const int *ctab = v.ctab + (size_t)v.hcell[i] * v.Mcap; // the masks index the culled table
    int q = 0, seen = 0;
    for (int w = 0; q < nb; ++w) {
        const unsigned word = v.mask[(size_t)w * N + i];
        const int cnt = __popc(word);
        while (q < nb && S[q] < seen + cnt) {
            out_j[(size_t)i * v.p + q] = ctab[(w << 5) + select_bit(word, S[q] - seen)];
            ++q;
        }
        seen += cnt;
    }
    out_n[i] = nb;
}

// g(r) counts: every pair once per ordered (i, j), classified like the force;
// hist[r][nbins] per replica.
__global__ void k_rdf(View v, float dr, int nbins, unsigned long long *hist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    bool live;
    const int r = slot_replica(v, i, live);
    if (!live) return;
    const size_t N = (size_t)v.N;
    const int4 pi = v.pos[i];
    const float h[3] = {v.box[r].h[0], v.box[r].h[1], v.box[r].h[2]};
    unsigned long long *hr = hist + (size_t)r * nbins;
    auto count = [&](int j, bool core_part) {
        PairGeom g = pair_geom(pi, v.pos[j], h);
        bool in;
        if (v.full_list) in = g.r2 < v.t_rs2;
        else in = core_part ? g.r2 < v.t_rc2 : (g.r2 >= v.t_rc2 && g.r2 < v.t_rs2);
        if (!in) return;
        float qf = __fdiv_rn(__fsqrt_rn(g.r2), dr);
        if (qf < (float)nbins) atomicAdd(&hr[(int)qf], 1ull);
    };
    if (v.full_list) { // explicit row-major rows
        const int n = min(v.n_shell[i], v.cap_c);
        for (int k = 0; k < n; ++k) count(v.core[(size_t)i * (size_t)v.cap_c + k], false);
        return;
    }
    {
        int nc = min(v.n_core[i], v.cap_c);
        for (int k = 0; k < nc; ++k) count(v.core[(size_t)k * N + i], true);
    }
    SegCursor cur;
    const int4 *tab = v.seg_tab + (size_t)v.hcell[i] * v.S;
    cur.init(tab);
    if (v.sampling) {
        // the stencil pool holds every pair with r < r_s outside the core
        const int self = pool_self_position(v.box[r], tab, i);
        const int M = tab[v.S - 1].w;
        for (int c = 0; c < M; ++c)
            if (c != self) count(cur.index_of(c), false);
        return;
    }
    const int *ctab = v.ctab + (size_t)v.hcell[i] * v.Mcap; // the masks index the culled table
    int left = v.n_shell[i];
    for (int w = 0; left > 0; ++w) {
        unsigned word = v.mask[(size_t)w * N + i];
        left -= __popc(word);
        while (word) {
            int bit = __ffs(word) - 1;
            word &= word - 1u;
            count(ctab[(w << 5) + bit], false);
        }
    }
}


} // namespace

cudaError_t launch_force_kernel(const View &v, int step_offset, bool energy, cudaStream_t s, bool prepare)
{
    if (v.potential == RBL_POT_LJ_EWALD) return launch_force_kernel_ewald(v, step_offset, energy, s, prepare);
    return launch_force_dispatch<false>(v, step_offset, energy, s, prepare);
}

cudaError_t launch_force_finish(const View &v, int advance, bool energy, cudaStream_t s)
{
    bool fp32 = v.precision == RBL_FP32;
    // FP64 force and energy sums are reduced from per-group partials; the FP32 path's
    // are exact integers already
    if (!fp32) k_force_chunks<<<dim3(v.pchunks, v.R), kChunkGroups, 0, s>>>(v);
    k_force_finish<<<v.R, fp32 ? 32 : kBlock, 0, s>>>(v, fp32 ? 1 : 0, (energy || !fp32) ? 1 : 0, v.subtract, advance,
                                                      0);
    return cudaGetLastError();
}

cudaError_t launch_exact_energy(const View &v, cudaStream_t s)
{
    cudaError_t e = v.potential == RBL_POT_LJ_EWALD ? launch_exact_energy_kernel_ewald(v, s)
                                                    : launch_exact_dispatch<false>(v, s);
    if (e != cudaSuccess) return e;
    k_force_chunks<<<dim3(v.pchunks, v.R), kChunkGroups, 0, s>>>(v);
    k_force_finish<<<v.R, kBlock, 0, s>>>(v, 0, 1, 0, 0, 1);
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

cudaError_t launch_batch(const View &v, unsigned long long step, int *out_j, int *out_n, cudaStream_t s)
{
    k_batch<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, step, out_j, out_n);
    return cudaGetLastError();
}

cudaError_t launch_rdf(const View &v, float dr, int nbins, unsigned long long *hist, cudaStream_t s)
{
    k_rdf<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, dr, nbins, hist);
    return cudaGetLastError();
}

} // namespace rbl
