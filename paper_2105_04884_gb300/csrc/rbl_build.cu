// rbl_build.cu -- linked cells and two-level neighbour lists (Sec. 2, Fig. 1).
//
// A rebuild is: cell hash + occupancy count (K1), exclusive scan of the counts,
// scatter into cell order and a per-cell sort by (x image, tag) (K2), permutation
// of the particle state into that order, and the list build (K3).  One launch per
// kernel covers every replica of the context.  Every kernel takes a `conditional`
// flag: in the stepping loop the chain runs only when the integrator raised some
// replica's device flag, and then each kernel leaves the particles and cells of
// replicas whose own flag is down untouched (their counts, order and lists stay
// valid, and the one scan over all cells reproduces their starts), so replicas
// rebuild exactly when they would on their own.
#include "rbl_internal.cuh"

namespace rbl {

namespace {

// Whole-kernel early exit: no replica is due.
__device__ __forceinline__ bool skip(const View &v, int conditional)
{
    return conditional && v.sc->rebuild == 0;
}

// Replica r takes part in this rebuild.
__device__ __forceinline__ bool active(const View &v, int conditional, int r)
{
    return !conditional || v.rs[r].rebuild != 0;
}

// Particle slot i that holds a particle of a rebuilding replica; r its replica.
__device__ __forceinline__ bool active_slot(const View &v, int conditional, int i, int &r)
{
    if (i >= v.N) return false;
    bool live;
    r = slot_replica(v, i, live);
    return live && active(v, conditional, r);
}

// Zero the occupancy counters (the pad cell of a replica holds its padding slots)
// and the build statistics of the rebuilding replicas.
__global__ void k_zero(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int stride = gridDim.x * blockDim.x;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.ncell; c += stride) {
        const int r = v.cell_rep[c];
        if (!active(v, conditional, r)) continue;
        const Box &b = v.box[r];
        v.counts[c] = c == b.c0 + b.ncell ? b.slots - b.N : 0;
        v.fill[c] = 0;
    }
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < v.R; r += stride) {
        if (!active(v, conditional, r)) continue;
        RepScalars &q = v.rs[r];
        q.nc_max = 0;
        q.ns_max = 0;
        q.m_max = 0;
        q.t_max = 0;
        q.ns_sum = 0ull;
        q.nc_sum = 0ull;
        q.m_sum = 0ull;
    }
}

// K1: cell of every particle from its fixed-point image, c_a = floor(u_a n_a / 2^32).
__global__ void k_cell_hash(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x, r;
    if (!active_slot(v, conditional, i, r)) return;
    const Box &b = v.box[r];
    int4 p = v.pos[i];
    int cx = cell_coord((unsigned)p.x, b.n[0]);
    int cy = cell_coord((unsigned)p.y, b.n[1]);
    int cz = cell_coord((unsigned)p.z, b.n[2]);
    int c = b.c0 + (cz * b.n[1] + cy) * b.n[0] + cx;
    v.cell[i] = c;
    atomicAdd(&v.counts[c], 1);
}

// Exclusive scan of counts -> start, in three passes: 2048-element tiles, the tile
// totals, and the tile offsets.
constexpr int kScanTile = 2048;

__device__ __forceinline__ int warp_incl_scan(int x)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    return x;
}

// Block-wide exclusive scan of one value per thread (blockDim.x multiple of 32, <= 1024).
__device__ int block_excl_scan(int x, int *total)
{
    __shared__ int warp_tot[32];
    __shared__ int block_tot;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = warp_incl_scan(x);
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
        int ti = warp_incl_scan(t);
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) block_tot = ti;
    }
    __syncthreads();
    int res = incl - x + warp_tot[wid];
    if (total) *total = block_tot;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(256) k_scan_tiles(View v, int conditional)
{
    if (skip(v, conditional)) return;
    constexpr int kPer = kScanTile / 256;
    int base = blockIdx.x * kScanTile + threadIdx.x * kPer;
    int vals[kPer];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        int c = base + k;
        vals[k] = c < v.ncell ? v.counts[c] : 0;
        sum += vals[k];
    }
    int total;
    int off = block_excl_scan(sum, &total);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        int c = base + k;
        if (c < v.ncell) v.start[c] = off;
        off += vals[k];
    }
    if (threadIdx.x == 0) v.blocksums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_totals(View v, int ntiles, int conditional)
{
    if (skip(v, conditional)) return;
    int per = (ntiles + 1023) / 1024;
    int base = threadIdx.x * per;
    int sum = 0;
    for (int k = 0; k < per; ++k)
        if (base + k < ntiles) sum += v.blocksums[base + k];
    int total;
    int off = block_excl_scan(sum, &total);
    for (int k = 0; k < per; ++k) {
        if (base + k < ntiles) {
            int t = v.blocksums[base + k];
            v.blocksums[base + k] = off;
            off += t;
        }
    }
    if (threadIdx.x == 0) v.start[v.ncell] = total;
}

__global__ void k_scan_add(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < v.ncell) v.start[c] += v.blocksums[c / kScanTile];
}

// K2a: scatter particle indices into their cell's slot range (arbitrary order
// within a cell; fixed by k_sort_cells).
__global__ void k_scatter(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x, r;
    if (!active_slot(v, conditional, i, r)) return;
    int c = v.cell[i];
    int slot = v.start[c] + atomicAdd(&v.fill[c], 1);
    v.order[slot] = i;
}

// K2b: order every cell's members by (x image, tag): insertion sort on packed
// (u_x, tag) keys carrying the index, in local memory for the usual small cells
// and in place in global memory for larger ones (no occupancy limit).
__global__ void k_sort_cells(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= v.ncell) return;
    const int r = v.cell_rep[c];
    if (!active(v, conditional, r) || c == v.box[r].c0 + v.box[r].ncell) return; // pad cell: no particles
    int s = v.start[c], e = v.start[c + 1];
    int m = e - s;
    auto key_of = [&](int idx) -> unsigned long long {
        int4 p = v.pos[idx];
        return ((unsigned long long)(unsigned)p.x << 32) | (unsigned)p.w;
    };
    if (m <= kCellCap) {
        unsigned long long key[kCellCap];
        int val[kCellCap];
        for (int k = 0; k < m; ++k) {
            val[k] = v.order[s + k];
            key[k] = key_of(val[k]);
        }
        for (int a = 1; a < m; ++a) {
            unsigned long long x = key[a];
            int xv = val[a];
            int b = a - 1;
            while (b >= 0 && key[b] > x) {
                key[b + 1] = key[b];
                val[b + 1] = val[b];
                --b;
            }
            key[b + 1] = x;
            val[b + 1] = xv;
        }
        for (int k = 0; k < m; ++k) v.order[s + k] = val[k];
    } else {
        int *o = v.order + s;
        for (int a = 1; a < m; ++a) {
            int x = o[a];
            unsigned long long kx = key_of(x);
            int b = a - 1;
            while (b >= 0 && key_of(o[b]) > kx) {
                o[b + 1] = o[b];
                --b;
            }
            o[b + 1] = x;
        }
    }
}

// Permute the state into cell order (into the alternate buffers) ...
__global__ void k_permute(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int k = blockIdx.x * blockDim.x + threadIdx.x, r;
    if (!active_slot(v, conditional, k, r)) return;
    int old = v.order[k];
    size_t N = (size_t)v.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v.x_alt[a * N + k] = v.x[a * N + old];
        v.v_alt[a * N + k] = v.v[a * N + old];
    }
    v.tag_alt[k] = v.tag[old];
    v.pos_alt[k] = v.pos[old];
}

// ... and back into the primary buffers, recording the build-time image.
__global__ void k_copy_back(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int k = blockIdx.x * blockDim.x + threadIdx.x, r;
    if (!active_slot(v, conditional, k, r)) return;
    size_t N = (size_t)v.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v.x[a * N + k] = v.x_alt[a * N + k];
        v.v[a * N + k] = v.v_alt[a * N + k];
    }
    const int t = v.tag_alt[k];
    v.tag[k] = t;
    int4 p = v.pos_alt[k];
    v.pos[k] = p;
    v.ubuild[k] = p;
    if (v.q) { // charges follow their particles
        const double qk = v.q_in[v.box[r].first + t];
        v.q[k] = qk;
        v.q32[k] = __double2float_rn(qk);
    }
}

// Prologue of the list builds: the home cell's candidate segments (warp-shared starts
// sA, lA of piece A and sB of piece B, running counts pre[0..S]) and the cell's
// seg_tab row.  Returns M_c, the candidate count.
__device__ __forceinline__ int cell_segments(const View &v, const Box &b, int c, int lc, int lane, int *pre, int *sA,
                                             int *lA, int *sB)
{
    const int S = b.S;
    const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
    const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
    const int nofs0 = b.nofs[0], nofs1 = b.nofs[1];
    // segment lengths, lane k holding segments k and k + 32 (S <= kMaxSeg < 64), then
    // their running counts by a warp scan
    int len2[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int sg = lane + 32 * h;
        if (sg < S) {
            int oz = sg / nofs1, oy = sg - oz * nofs1;
            int czz = wrap_cell(cz + b.ofs[2][oz], n2);
            int cyy = wrap_cell(cy + b.ofs[1][oy], n1);
            int rowbase = b.c0 + (czz * n1 + cyy) * n0;
            int fx = wrap_cell(cx + b.ofs[0][0], n0);
            int last = fx + nofs0 - 1;
            int lastA = last < n0 ? last : n0 - 1;
            int a0 = v.start[rowbase + fx];
            int la = v.start[rowbase + lastA + 1] - a0;
            int b0 = v.start[rowbase];
            int lb = last >= n0 ? v.start[rowbase + (last - n0) + 1] - b0 : 0;
            sA[sg] = a0;
            lA[sg] = la;
            sB[sg] = b0;
            len2[h] = la + lb;
        }
    }
    int carry = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int x = len2[h];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        x += carry;
        const int sg = lane + 32 * h;
        if (sg < S) pre[sg + 1] = x;
        carry = __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) pre[0] = 0;
    __syncwarp();
    const int M = pre[S];
    int4 *gt = v.seg_tab + (size_t)c * v.S;
    for (int sg = lane; sg < v.S; sg += 32) {
        if (sg < S) {
            const int split = pre[sg] + lA[sg];
            gt[sg] = make_int4(sA[sg] - pre[sg], split, sB[sg] - split, pre[sg + 1]);
        } else {
            gt[sg] = make_int4(0, M, 0, M);
        }
    }
    return M;
}

// K3: the lists.  One warp per home cell: the warp takes candidates 32 at a time (one
// per lane, fetched once) and tests each against every particle of the cell:
//   core : r2 <  (r_c + skin)^2                         -> explicit list (ballot rank)
//   shell: max(r_c - skin, 0)^2 <= r2 < (r_s + skin)^2  -> mask word (ballot)
//   full : r2 <  (r_s + skin)^2   (full_list mode: explicit row-major rows, no mask)
// Candidates are visited in canonical order, so list order and bit order are the
// canonical row order.  Particle k of a pass of up to 32 keeps its counters in lane
// k.  Row lengths are counted past the core capacity.  k_build_pool serves the
// stencil pool (the paper's own pool), where only the core row is built, from the 27
// cells around the home cell, and a particle's pool size is its home cell's stencil
// population less itself (the segment table spans the whole stencil, for the batch);
// k_build_culled serves shell sampling and the full list, testing only the candidates
// that survive a cull against the cell's bounding box.
constexpr int kMaxBuildWarps = 8; // home cells (warps) per block: a launch parameter, 2, 4 or 8

// LIST (k_build_culled): kListShell (core row + shell mask) or kListFull (full-list
// rows), fixed at compile time so that the pair-test loop carries no mode branches.
enum { kListShell = 0, kListFull = 1 };

__global__ void __launch_bounds__(kMaxBuildWarps * 32) k_build_pool(View v, int conditional)
{
    if (skip(v, conditional)) return;
    __shared__ int s_pre[kMaxBuildWarps][kMaxSeg + 1];
    __shared__ int s_a[kMaxBuildWarps][kMaxSeg], s_la[kMaxBuildWarps][kMaxSeg], s_b[kMaxBuildWarps][kMaxSeg];
    __shared__ int4 s_pos[kMaxBuildWarps][32];
    __shared__ int s_j[kMaxBuildWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= v.ncell) return; // whole warp; no block-wide barrier below
    const int r = v.cell_rep[c];
    const Box &b = v.box[r];
    const int lc = c - b.c0;
    if (lc == b.ncell || !active(v, conditional, r)) return; // pad cell, or not rebuilding
    int *pre = s_pre[warp], *sA = s_a[warp], *lA = s_la[warp], *sB = s_b[warp];
    const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
    const int cx = lc % n0, cy = (lc / n0) % n1, cz = lc / (n0 * n1);
    const int S = b.S;
    const int M = cell_segments(v, b, c, lc, lane, pre, sA, lA, sB);
    const int s0 = v.start[c], s1 = v.start[c + 1];
    if (s1 == s0) return;
    // the masks index this cell's candidate sequence: remember the cell until the
    // next build, however far the particle drifts meanwhile
    for (int i = s0 + lane; i < s1; i += 32) v.hcell[i] = c;
    RepScalars &rsc = v.rs[r];
    const float h[3] = {b.h[0], b.h[1], b.h[2]};
    // Stencil-pool sampling: no shell rows; the core row comes from the cells within
    // one cell of the home cell (the cell edge is at least r_c + skin), taken in the
    // order they have in the full stencil, one single-cell segment each.
    int Sseg = S, Mloop = M;
    {
        // near offsets per axis in the stencil's order: -1, 0, 1 (offsets relative to
        // the home cell), or 0, 1, n-1 (every cell once from the home cell; fewer
        // when n < 3); lane k takes near cell k, in z-major order, then one warp scan
        int nn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) nn[a] = b.ofs[a][0] < 0 ? 3 : min(b.n[a], 3);
        auto near_o = [&](int a, int k) { return b.ofs[a][0] < 0 ? k - 1 : (k < 2 ? k : b.n[a] - 1); };
        const int nseg = nn[0] * nn[1] * nn[2];
        int st = 0, len = 0;
        if (lane < nseg) {
            const int iz = lane / (nn[1] * nn[0]), iy = (lane / nn[0]) % nn[1], ix = lane % nn[0];
            const int cell = b.c0 + (wrap_cell(cz + near_o(2, iz), n2) * n1 + wrap_cell(cy + near_o(1, iy), n1)) * n0 +
                             wrap_cell(cx + near_o(0, ix), n0);
            st = v.start[cell];
            len = v.start[cell + 1] - st;
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        __syncwarp(); // every lane is done with the full-stencil segments
        if (lane < nseg) {
            sA[lane] = st;
            lA[lane] = len;
            sB[lane] = 0;
            pre[lane + 1] = incl;
        }
        if (lane == 0) pre[0] = 0;
        __syncwarp();
        Sseg = nseg;
        Mloop = pre[nseg];
    }
    const int nchunk = (Mloop + 31) >> 5;
    const size_t N = (size_t)v.N;
    int wmc = 0, wms = 0;
    unsigned long long wsc = 0ull, wss = 0ull;
    for (int base = s0; base < s1; base += 32) {
        const int mm = min(32, s1 - base);
        const int i_me = base + lane; // the particle this lane stores for (lane < mm)
        if (lane < mm) s_pos[warp][lane] = v.pos[i_me];
        __syncwarp();
        int my_nc = 0, my_ns = 0;
        int seg = 0;
        for (int k = 0; k < nchunk; ++k) {
            const int cand = (k << 5) + lane;
            const bool valid = cand < Mloop;
            int sg = seg;
            while (sg + 1 < Sseg && pre[sg + 1] <= cand) ++sg;
            const int off = cand - pre[sg];
            const int j = off < lA[sg] ? sA[sg] + off : sB[sg] + (off - lA[sg]);
            const int4 pj = valid ? v.pos[j] : make_int4(0, 0, 0, 0);
            seg = __shfl_sync(0xffffffffu, sg, 31);
            s_j[warp][lane] = j;
            // test the 32 candidates against each particle of the pass; lane q keeps
            // particle q's core word
            unsigned my_core = 0u;
            for (int q = 0; q < mm; ++q) {
                PairGeom g = pair_geom(s_pos[warp][q], pj, h);
                const bool other = valid && j != base + q;
                const bool in_core = other && g.r2 < v.t_core_list;
                const unsigned bc = __ballot_sync(0xffffffffu, in_core);
                my_core = lane == q ? bc : my_core;
            }
            __syncwarp();
            if (lane < mm) {
                while (my_core) { // core row in candidate order
                    const int b = __ffs(my_core) - 1;
                    my_core &= my_core - 1u;
                    if (my_nc < v.cap_c) v.core[(size_t)my_nc * N + i_me] = s_j[warp][b];
                    ++my_nc;
                }
            }
            __syncwarp();
        }
        if (lane < mm) {
            my_ns = M - 1; // the pool: every other particle of the stencil
            v.n_core[i_me] = my_nc;
            v.n_shell[i_me] = my_ns;
            if (my_nc > v.cap_c) atomicOr(&v.sc->flags, kFlagOverflow);
            wmc = max(wmc, my_nc);
            wms = max(wms, my_ns);
            wsc += (unsigned long long)my_nc;
            wss += (unsigned long long)my_ns;
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wmc = max(wmc, __shfl_xor_sync(0xffffffffu, wmc, o));
        wms = max(wms, __shfl_xor_sync(0xffffffffu, wms, o));
        wsc += __shfl_xor_sync(0xffffffffu, wsc, o);
        wss += __shfl_xor_sync(0xffffffffu, wss, o);
    }
    if (lane == 0) {
        atomicMax(&rsc.nc_max, wmc);
        atomicMax(&rsc.ns_max, wms);
        atomicMax(&rsc.m_max, M);
        atomicAdd(&rsc.nc_sum, wsc);
        atomicAdd(&rsc.ns_sum, wss);
        atomicAdd(&rsc.m_sum, (unsigned long long)M * (unsigned long long)(s1 - s0));
    }
}

// Culled list build (shell rows with their candidate table, or full rows).  One warp
// per home cell, as k_build_pool, with one step in front of the pair tests: each
// candidate (one per lane, fetched once) is first tested against the bounding box of
// the cell's particles, and only the candidates that some particle of the cell may
// reach go on, compacted in order into a ring of kRing entries; every 32 of them form
// one dense chunk that is tested against each particle of the pass with the
// canonical pair rule.  Dense chunk k is mask word k (shell mode) and entries
// 32k .. 32k + 31 of the cell's candidate table ctab, so masks index the table; the
// rows, which only ever hold candidates within r_s + skin, are those of the full
// candidate sequence.
//
// The cull is conservative.  Along axis a the box is the arc [c_a - hl_a, c_a + hh_a]
// of the periodic fixed-point circle (2^32 units) around its centre c_a; e_a, the
// candidate's offset from c_a as int32 (its minimum image), gives the circular gap
// g_a = max(0, e_a - hh_a, -e_a - hl_a), and |(int32)(u_i - u_j)|_a >= g_a for every
// particle i of the cell, in a box of any size.  The pair rule's r2 is then at least
// (1 - 2^-21) sum_a (g_a h_a)^2 (each of its six binary32 operations rounds by at
// most 2^-24), and the cull's own binary32 estimate of that sum (with hl, hh rounded
// up) exceeds it by less than 2^-20, so a candidate whose estimate is at least
// (r_s + skin)^2 (1 + 2^-12) is beyond the list cutoff for every particle.
constexpr int kRing = 64;

// Shared memory of one warp of k_build_culled (dynamic: build_warps of them per block).
struct CullWarpSmem {
    int4 rp[kRing];           // ring of kept candidates: images
    int4 pos[32];             // the pass's particles
    int rj[kRing];            // ring: particle indices
    int pre[kMaxSeg + 1], a[kMaxSeg], la[kMaxSeg], b[kMaxSeg]; // candidate segments
};

// 64 registers (four blocks of the largest shape per SM): measured faster than the
// unbounded 80 despite a few spilled bytes (316.7 against 353.7 us at N = 2^18).
template <int LIST>
__global__ void __launch_bounds__(kMaxBuildWarps * 32, 4) k_build_culled(View v, int conditional)
{
    if (skip(v, conditional)) return;
    extern __shared__ int4 s_cull[];
    constexpr bool full = LIST == kListFull;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CullWarpSmem &sm = reinterpret_cast<CullWarpSmem *>(s_cull)[warp];
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= v.ncell) return; // whole warp; no block-wide barrier below
    const int r = v.cell_rep[c];
    const Box &b = v.box[r];
    const int lc = c - b.c0;
    if (lc == b.ncell || !active(v, conditional, r)) return; // pad cell, or not rebuilding
    const int M = cell_segments(v, b, c, lc, lane, sm.pre, sm.a, sm.la, sm.b);
    const int S = b.S;
    const int s0 = v.start[c], s1 = v.start[c + 1];
    if (s1 == s0) return;
    for (int i = s0 + lane; i < s1; i += 32) v.hcell[i] = c;
    RepScalars &rsc = v.rs[r];
    const float h[3] = {b.h[0], b.h[1], b.h[2]};
    // bounding box of the cell's particles in fixed-point units relative to its first
    // particle (differences as int32: a cell spans less than half the box), then its
    // centre and half-widths, rounded up as binary32
    const int4 p0 = v.pos[s0];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int i = s0 + lane; i < s1; i += 32) {
        const int4 p = v.pos[i];
        const int d[3] = {(int)((unsigned)p.x - (unsigned)p0.x), (int)((unsigned)p.y - (unsigned)p0.y),
                          (int)((unsigned)p.z - (unsigned)p0.z)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], d[a]);
            hi[a] = max(hi[a], d[a]);
        }
    }
    unsigned cen[3];
    float hlf[3], hhf[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        const int mid = lo[a] + ((hi[a] - lo[a]) >> 1);
        cen[a] = (a == 0 ? (unsigned)p0.x : a == 1 ? (unsigned)p0.y : (unsigned)p0.z) + (unsigned)mid;
        hlf[a] = __int2float_ru(mid - lo[a]);
        hhf[a] = __int2float_ru(hi[a] - mid);
    }
    int *ctab_c = v.ctab + (size_t)c * v.Mcap;
    const size_t N = (size_t)v.N;
    const unsigned lt_mask = (1u << lane) - 1u;
    int wmc = 0, wms = 0;
    unsigned long long wsc = 0ull, wss = 0ull;
    for (int base = s0; base < s1; base += 32) {
        const int mm = min(32, s1 - base);
        const int i_me = base + lane; // the particle this lane stores for (lane < mm)
        if (lane < mm) sm.pos[lane] = v.pos[i_me];
        __syncwarp();
        int my_nc = 0, my_ns = 0;
        int head = 0, tail = 0, kd = 0;
        // one dense chunk: ring entries head .. head + nd - 1 against every particle
        // of the pass (mask word kd, table entries 32 kd ..)
        auto dense = [&](int nd) {
            const bool dv = lane < nd;
            const int slot = (head + lane) & (kRing - 1);
            const int jd = sm.rj[slot];
            const int4 pd = sm.rp[slot];
            const bool room = full || kd < v.W; // table and masks hold W words' worth
            if (!full && base == s0 && dv && room) ctab_c[(kd << 5) + lane] = jd;
            unsigned my_shell = 0u, my_core = 0u;
            for (int q = 0; q < mm; ++q) {
                PairGeom g = pair_geom(sm.pos[q], pd, h);
                const bool other = dv && jd != base + q;
                if constexpr (full) {
                    const bool in = other && g.r2 < v.t_cut_list;
                    const unsigned bf = __ballot_sync(0xffffffffu, in);
                    const int n0q = __shfl_sync(0xffffffffu, my_nc, q);
                    if (in) {
                        const int rk = n0q + __popc(bf & lt_mask);
                        if (rk < v.cap_c) v.core[(size_t)(base + q) * (size_t)v.cap_c + rk] = jd;
                    }
                    if (lane == q) my_nc += __popc(bf);
                } else {
                    const bool in_shell = other && g.r2 >= v.t_shell_lo && g.r2 < v.t_cut_list;
                    const unsigned bs = __ballot_sync(0xffffffffu, in_shell);
                    my_shell = lane == q ? bs : my_shell;
                    const bool in_core = other && g.r2 < v.t_core_list;
                    const unsigned bc = __ballot_sync(0xffffffffu, in_core);
                    my_core = lane == q ? bc : my_core;
                }
            }
            if (lane < mm && !full && room) {
                v.mask[(size_t)kd * N + i_me] = my_shell; // coalesced across lanes
                my_ns += __popc(my_shell);
                while (my_core) { // core row in candidate order
                    const int bb = __ffs(my_core) - 1;
                    my_core &= my_core - 1u;
                    if (my_nc < v.cap_c) v.core[(size_t)my_nc * N + i_me] = sm.rj[(head + bb) & (kRing - 1)];
                    ++my_nc;
                }
            }
            __syncwarp();
            head += nd;
            ++kd;
        };
        // the candidates segment by segment (each a run of particle indices in one or
        // two pieces), 32 at a time: cull, append the kept ones to the ring in order,
        // and test every full chunk of 32 as soon as it is there
        for (int sg = 0; sg < S; ++sg) {
            const int a0 = sm.a[sg], la = sm.la[sg], b0 = sm.b[sg];
            const int n_sg = sm.pre[sg + 1] - sm.pre[sg];
            for (int o0 = 0; o0 < n_sg; o0 += 32) {
                const int off = o0 + lane;
                bool keep = false;
                int j = 0;
                int4 pj = make_int4(0, 0, 0, 0);
                if (off < n_sg) {
                    j = off < la ? a0 + off : b0 + (off - la);
                    pj = v.pos[j];
                    const int e[3] = {(int)((unsigned)pj.x - cen[0]), (int)((unsigned)pj.y - cen[1]),
                                      (int)((unsigned)pj.z - cen[2])};
                    float g2 = 0.f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float ef = __int2float_rn(e[a]);
                        const float gap = fmaxf(0.f, fmaxf(__fsub_rn(ef, hhf[a]), __fsub_rn(-ef, hlf[a])));
                        const float ga = __fmul_rn(gap, h[a]);
                        g2 = __fmaf_rn(ga, ga, g2);
                    }
                    keep = g2 < v.t_cull;
                }
                const unsigned kb = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int slot = (tail + __popc(kb & lt_mask)) & (kRing - 1);
                    sm.rj[slot] = j;
                    sm.rp[slot] = pj;
                }
                tail += __popc(kb);
                __syncwarp();
                if (tail - head >= 32) dense(32); // at most one: fewer than 32 were pending
            }
        }
        if (tail > head) dense(tail - head);
        if (!full && base == s0 && lane == 0) v.ctab_n[c] = tail;
        if (!full && tail > v.Mcap) {
            // the culled table outgrew its capacity: flag it and leave these particles
            // with empty rows, so that no kernel decodes a mask that was not written
            my_nc = my_ns = 0;
            if (lane == 0) atomicOr(&v.sc->flags, kFlagCellOverflow);
        }
        if (lane == 0) atomicMax(&rsc.t_max, tail);
        if (lane < mm) {
            if (full) { // the full row's length, counted as the shell's
                my_ns = my_nc;
                my_nc = 0;
                if (my_ns > v.cap_c) atomicOr(&v.sc->flags, kFlagOverflow);
            }
            v.n_core[i_me] = my_nc;
            v.n_shell[i_me] = my_ns;
            if (my_nc > v.cap_c) atomicOr(&v.sc->flags, kFlagOverflow);
            wmc = max(wmc, my_nc);
            wms = max(wms, my_ns);
            wsc += (unsigned long long)my_nc;
            wss += (unsigned long long)my_ns;
        }
        __syncwarp();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wmc = max(wmc, __shfl_xor_sync(0xffffffffu, wmc, o));
        wms = max(wms, __shfl_xor_sync(0xffffffffu, wms, o));
        wsc += __shfl_xor_sync(0xffffffffu, wsc, o);
        wss += __shfl_xor_sync(0xffffffffu, wss, o);
    }
    if (lane == 0) {
        atomicMax(&rsc.nc_max, wmc);
        atomicMax(&rsc.ns_max, wms);
        atomicMax(&rsc.m_max, M);
        atomicAdd(&rsc.nc_sum, wsc);
        atomicAdd(&rsc.ns_sum, wss);
        atomicAdd(&rsc.m_sum, (unsigned long long)M * (unsigned long long)(s1 - s0));
    }
}

// Graph form of the rebuild decision: set the conditional node's value from the
// device flag the integrator raised.
__global__ void k_set_condition(View v, cudaGraphConditionalHandle h)
{
    cudaGraphSetConditional(h, v.sc->rebuild ? 1u : 0u);
}

__global__ void k_finish(View v, int conditional)
{
    if (skip(v, conditional)) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < v.R && active(v, conditional, r)) {
        v.rs[r].rebuild = 0;
        v.rs[r].n_rebuild += 1;
    }
}

// Runs after k_finish: the context-wide flag is cleared only once every replica
// has read it.
__global__ void k_finish_all(View v) { v.sc->rebuild = 0; }

} // namespace

cudaError_t launch_rebuild_sort(const View &v, int n_scan_blocks, bool conditional, cudaStream_t s)
{
    int cond = conditional ? 1 : 0;
    int gN = ceil_div(v.N, kBlock);
    int gC = ceil_div(v.ncell, kBlock);
    int gZ = gC < 1024 ? gC : 1024;
    k_zero<<<gZ, kBlock, 0, s>>>(v, cond);
    k_cell_hash<<<gN, kBlock, 0, s>>>(v, cond);
    k_scan_tiles<<<n_scan_blocks, 256, 0, s>>>(v, cond);
    k_scan_totals<<<1, 1024, 0, s>>>(v, n_scan_blocks, cond);
    k_scan_add<<<gC, kBlock, 0, s>>>(v, cond);
    k_scatter<<<gN, kBlock, 0, s>>>(v, cond);
    k_sort_cells<<<gC, kBlock, 0, s>>>(v, cond);
    k_permute<<<gN, kBlock, 0, s>>>(v, cond);
    k_copy_back<<<gN, kBlock, 0, s>>>(v, cond);
    return cudaGetLastError();
}

cudaError_t launch_rebuild_lists(const View &v, bool conditional, cudaStream_t s)
{
    int cond = conditional ? 1 : 0;
    const dim3 gB(ceil_div(v.ncell, v.build_warps)), bB(v.build_warps * 32);
    const size_t smem = sizeof(CullWarpSmem) * (size_t)v.build_warps;
    if (v.sampling) k_build_pool<<<gB, bB, 0, s>>>(v, cond);
    else if (v.full_list) k_build_culled<kListFull><<<gB, bB, smem, s>>>(v, cond);
    else k_build_culled<kListShell><<<gB, bB, smem, s>>>(v, cond);
    k_finish<<<ceil_div(v.R, kBlock), kBlock, 0, s>>>(v, cond);
    k_finish_all<<<1, 1, 0, s>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const View &v, int n_scan_blocks, bool conditional, cudaStream_t s)
{
    cudaError_t e = launch_rebuild_sort(v, n_scan_blocks, conditional, s);
    if (e == cudaSuccess) e = launch_rebuild_lists(v, conditional, s);
    return e;
}

cudaError_t launch_set_rebuild_condition(const View &v, cudaGraphConditionalHandle h, cudaStream_t s)
{
    k_set_condition<<<1, 1, 0, s>>>(v, h);
    return cudaGetLastError();
}

} // namespace rbl
