// rbl_build.cu -- linked cells and two-level neighbour lists (Sec. 2, Fig. 1).
//
// A rebuild is: cell hash + occupancy count (K1), exclusive scan of the counts,
// scatter into cell order and a per-cell sort by tag (K2), permutation of the
// particle state into that order, and the list build (K3).  Every kernel takes a
// `conditional` flag: in the stepping loop the rebuild is enqueued every step and
// each kernel returns at once unless the integrator raised the device flag
// DevScalars::rebuild, so no host round trip decides whether to rebuild.
#include "rbl_internal.cuh"

namespace rbl {

namespace {

__device__ __forceinline__ bool skip(const View &v, int conditional)
{
    return conditional && v.sc->rebuild == 0;
}

// Zero the occupancy counters and the build statistics.
__global__ void k_zero(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int stride = gridDim.x * blockDim.x;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < v.ncell; c += stride) {
        v.counts[c] = 0;
        v.fill[c] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        v.sc->nc_max = 0;
        v.sc->ns_max = 0;
        v.sc->ns_sum = 0ull;
        v.sc->nc_sum = 0ull;
    }
}

// K1: cell of every particle from its fixed-point image, c_a = floor(u_a n_a / 2^32).
__global__ void k_cell_hash(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    int4 p = v.pos[i];
    int cx = cell_coord((unsigned)p.x, v.n[0]);
    int cy = cell_coord((unsigned)p.y, v.n[1]);
    int cz = cell_coord((unsigned)p.z, v.n[2]);
    int c = (cz * v.n[1] + cy) * v.n[0] + cx;
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
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.N) return;
    int c = v.cell[i];
    int slot = v.start[c] + atomicAdd(&v.fill[c], 1);
    v.order[slot] = i;
}

// K2b: order every cell's members by tag: insertion sort on packed (tag, index)
// keys, in registers/local memory for the usual small cells and in place in global
// memory for larger ones (no occupancy limit).
__global__ void k_sort_cells(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= v.ncell) return;
    int s = v.start[c], e = v.start[c + 1];
    int m = e - s;
    if (m <= kCellCap) {
        unsigned long long key[kCellCap];
        for (int k = 0; k < m; ++k) {
            int idx = v.order[s + k];
            key[k] = ((unsigned long long)(unsigned)v.tag[idx] << 32) | (unsigned)idx;
        }
        for (int a = 1; a < m; ++a) {
            unsigned long long x = key[a];
            int b = a - 1;
            while (b >= 0 && key[b] > x) {
                key[b + 1] = key[b];
                --b;
            }
            key[b + 1] = x;
        }
        for (int k = 0; k < m; ++k) v.order[s + k] = (int)(unsigned)key[k];
    } else {
        int *o = v.order + s;
        for (int a = 1; a < m; ++a) {
            int x = o[a];
            int tx = v.tag[x];
            int b = a - 1;
            while (b >= 0 && v.tag[o[b]] > tx) {
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
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.N) return;
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
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.N) return;
    size_t N = (size_t)v.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v.x[a * N + k] = v.x_alt[a * N + k];
        v.v[a * N + k] = v.v_alt[a * N + k];
    }
    v.tag[k] = v.tag_alt[k];
    int4 p = v.pos_alt[k];
    v.pos[k] = p;
    v.ubuild[k] = p;
}

__device__ __forceinline__ int wrap_cell(int c, int n)
{
    c %= n;
    return c < 0 ? c + n : c;
}

// K3: two-level lists (or the full list).  One thread per particle walks the
// stencil in canonical order (z-major, x-minor slots; members of a cell in tag
// order) and appends every neighbour inside a window:
//   core : r2 <  (r_c + skin)^2
//   shell: max(r_c - skin, 0)^2 <= r2 < (r_s + skin)^2
//   full : r2 <  (r_s + skin)^2          (full_list mode, stored in the shell rows)
// Lengths are counted past the capacity so the caller learns the size needed.
__global__ void __launch_bounds__(kBlock) k_build_lists(View v, int conditional)
{
    if (skip(v, conditional)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int nc = 0, ns = 0;
    if (i < v.N) {
        int4 pi = v.pos[i];
        int ci[3] = {cell_coord((unsigned)pi.x, v.n[0]), cell_coord((unsigned)pi.y, v.n[1]),
                     cell_coord((unsigned)pi.z, v.n[2])};
        int *crow = v.core + (size_t)i * v.cap_c;
        int *srow = v.shell + (size_t)i * v.cap_s;
        const bool full = v.full_list != 0;
        for (int oz = 0; oz < v.nofs[2]; ++oz) {
            int cz = wrap_cell(ci[2] + v.ofs[2][oz], v.n[2]);
            for (int oy = 0; oy < v.nofs[1]; ++oy) {
                int cy = wrap_cell(ci[1] + v.ofs[1][oy], v.n[1]);
                int rowbase = (cz * v.n[1] + cy) * v.n[0];
                for (int ox = 0; ox < v.nofs[0]; ++ox) {
                    int c = rowbase + wrap_cell(ci[0] + v.ofs[0][ox], v.n[0]);
                    int s = v.start[c], e = v.start[c + 1];
                    for (int j = s; j < e; ++j) {
                        if (j == i) continue;
                        PairGeom g = pair_geom(pi, v.pos[j], v.h);
                        if (full) {
                            if (g.r2 < v.t_cut_list) {
                                if (ns < v.cap_s) srow[ns] = j;
                                ++ns;
                            }
                        } else {
                            if (g.r2 < v.t_core_list) {
                                if (nc < v.cap_c) crow[nc] = j;
                                ++nc;
                            }
                            if (g.r2 >= v.t_shell_lo && g.r2 < v.t_cut_list) {
                                if (ns < v.cap_s) srow[ns] = j;
                                ++ns;
                            }
                        }
                    }
                }
            }
        }
        v.n_core[i] = nc;
        v.n_shell[i] = ns;
        if (nc > v.cap_c || ns > v.cap_s) atomicOr(&v.sc->flags, kFlagOverflow);
    }
    // row statistics
    int mc = nc, ms = ns;
    unsigned long long ss = (unsigned long long)ns, cs = (unsigned long long)nc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        ms = max(ms, __shfl_xor_sync(0xffffffffu, ms, o));
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        cs += __shfl_xor_sync(0xffffffffu, cs, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&v.sc->nc_max, mc);
        atomicMax(&v.sc->ns_max, ms);
        atomicAdd(&v.sc->ns_sum, ss);
        atomicAdd(&v.sc->nc_sum, cs);
    }
}

__global__ void k_finish(View v, int conditional)
{
    if (skip(v, conditional)) return;
    v.sc->rebuild = 0;
    v.sc->n_rebuild += 1;
}

} // namespace

cudaError_t launch_rebuild(const View &v, int n_scan_blocks, bool conditional, cudaStream_t s)
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
    k_build_lists<<<gN, kBlock, 0, s>>>(v, cond);
    k_finish<<<1, 1, 0, s>>>(v, cond);
    return cudaGetLastError();
}

} // namespace rbl
