// rbl_capi.cu -- host side of the C ABI declared in include/rbl.h.
//
// The context lives in host memory; every device array is carved out of the
// caller's workspace.  A context holds R >= 1 independent replicas (rbl_create
// makes R = 1); each kernel launch covers all of them.  A step of Algorithm 1 is
// enqueued as: fused kick/drift/thermostat kernel, the (device-conditional)
// rebuild chain, the force kernel and its reduction.  The steady-state step is
// captured once in a CUDA graph and replayed; the step counter lives in device
// memory so replays stay valid.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "rbl_internal.cuh"

using namespace rbl;

namespace {

const double kPi = 3.14159265358979323846264338327950288;
constexpr long long kMaxSlots = 1ll << 30;  // particle slots of a context (int indices, int32 rows)

// Sizes and offsets of every array of a context's workspace.
struct Plan {
    size_t off[40];
    int n;
    size_t total;
    int R, N, ntile, ncell, cap_c, W, S, Mcap, n_scan_blocks, pchunks;
    long long n_real;
    size_t staging_bytes;
};

// Cell grid and candidate statistics of one replica.
struct Geo {
    int n3[3], nofs3[3], S, ncell, mcap;
    double core_mean;  // mean core row (r < r_c + skin)
    double full_mean;  // mean full row (r < r_s + skin)
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int round_up(int x, int m) { return (x + m - 1) / m * m; }

long long round_up_ll(long long x, long long m) { return (x + m - 1) / m * m; }

void set_err(rbl_ctx *c, const char *fmt, ...)
{
    if (!c) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
}

#define BAD(...)                                       \
    do {                                               \
        if (err) snprintf(err, errlen, __VA_ARGS__);   \
        return RBL_EINVAL;                             \
    } while (0)

rbl_status validate(const rbl_params *p, int N, char *err, size_t errlen)
{
    if (!p) BAD("params is NULL");
    if (N < 2) BAD("N must be >= 2 (got %d)", N);
    const double vals[] = {p->L[0], p->L[1], p->L[2], p->r_c, p->r_s, p->skin, p->dt, p->T, p->gamma, p->rho_cap,
                           p->alpha};
    for (double v : vals)
        if (!std::isfinite(v)) BAD("non-finite parameter");
    if (!(p->r_c > 0.0 && p->r_c < p->r_s)) BAD("need 0 < r_c < r_s (got r_c=%g, r_s=%g)", p->r_c, p->r_s);
    if (!(p->skin >= 0.0)) BAD("skin must be >= 0");
    if (p->p < 1 || p->p > kMaxP) BAD("p must be in 1..%d (got %d)", kMaxP, p->p);
    if (!(p->dt > 0.0)) BAD("dt must be > 0");
    if (!(p->T >= 0.0) || !(p->gamma >= 0.0)) BAD("T and gamma must be >= 0");
    if (p->cells_per_cutoff < 1 || p->cells_per_cutoff > 3) BAD("cells_per_cutoff must be 1..3");
    if (p->precision != RBL_FP32 && p->precision != RBL_FP64) BAD("precision must be RBL_FP32 or RBL_FP64");
    for (int a = 0; a < 3; ++a)
        if (!(p->L[a] >= 2.0 * (p->r_s + p->skin)))
            BAD("box length L[%d]=%g is below 2 (r_s + skin) = %g", a, p->L[a], 2.0 * (p->r_s + p->skin));
    if (p->cap_core < 0 || p->cap_stencil < 0 || !(p->rho_cap >= 0.0)) BAD("capacities must be >= 0");
    if (p->sampling != RBL_SAMPLE_SHELL && p->sampling != RBL_SAMPLE_STENCIL)
        BAD("sampling must be RBL_SAMPLE_SHELL or RBL_SAMPLE_STENCIL");
    if (p->potential != RBL_POT_LJ && p->potential != RBL_POT_LJ_EWALD)
        BAD("potential must be RBL_POT_LJ or RBL_POT_LJ_EWALD");
    if (p->potential == RBL_POT_LJ_EWALD && !(p->alpha > 0.0)) BAD("RBL_POT_LJ_EWALD needs alpha > 0");
    if (p->sampling == RBL_SAMPLE_STENCIL) {
        if (p->full_list) BAD("stencil-pool sampling is an RBL mode: full_list must be 0");
        if (2 * ((int)std::floor(p->r_s / p->r_c) + 1) + 1 > kMaxStencil)
            BAD("stencil-pool sampling needs r_s / r_c < 3 (got %g)", p->r_s / p->r_c);
    }
    double cells = 1.0;
    for (int a = 0; a < 3; ++a) cells *= std::floor(p->L[a] * p->cells_per_cutoff / (p->r_s + p->skin));
    if (cells > (double)(1 << 28)) BAD("box too large: %.0f cells", cells);
    return RBL_OK;
}

// Replicas share everything but the box, the temperature, the seed and N.
rbl_status validate_batch(const rbl_params *prm, int R, const int *N, char *err, size_t errlen)
{
    if (!prm || !N || R < 1) BAD("need R >= 1 replicas with params and sizes (got R=%d)", R);
    long long slots = 0;
    for (int r = 0; r < R; ++r) {
        rbl_status st = validate(&prm[r], N[r], err, errlen);
        if (st != RBL_OK) return st;
        const rbl_params &a = prm[0], &b = prm[r];
        if (a.r_c != b.r_c || a.r_s != b.r_s || a.skin != b.skin || a.p != b.p || a.dt != b.dt ||
            a.gamma != b.gamma || a.precision != b.precision || a.full_list != b.full_list ||
            a.subtract_net_force != b.subtract_net_force || a.cells_per_cutoff != b.cells_per_cutoff ||
            a.cap_core != b.cap_core || a.cap_stencil != b.cap_stencil || a.rho_cap != b.rho_cap ||
            a.sampling != b.sampling || a.potential != b.potential || a.alpha != b.alpha)
            BAD("replica %d differs from replica 0 in a shared parameter (only L, T, seed may differ)", r);
        slots += round_up_ll(N[r], kTile);
    }
    if (slots > kMaxSlots) BAD("too many particles: %lld slots (limit %lld)", slots, kMaxSlots);
    return RBL_OK;
}
#undef BAD

Geo replica_geo(const rbl_params *p, int N)
{
    Geo g{};
    const double rho = p->rho_cap > 0.0 ? p->rho_cap : N / (p->L[0] * p->L[1] * p->L[2]);
    // shell sampling: cells of width >= (r_s + skin) / K, stencil half-width K;
    // stencil pool: cells of edge >= r_c + skin, half-width floor(r_s / r_c) + 1
    const bool pool = p->sampling == RBL_SAMPLE_STENCIL;
    const int K = pool ? (int)std::floor(p->r_s / p->r_c) + 1 : p->cells_per_cutoff;
    long long nc = 1;
    double span = 1.0;
    for (int a = 0; a < 3; ++a) {
        int n = pool ? (int)std::floor(p->L[a] / (p->r_c + p->skin))
                     : (int)std::floor(p->L[a] * (double)p->cells_per_cutoff / (p->r_s + p->skin));
        if (n < 1) n = 1;
        g.n3[a] = n;
        g.nofs3[a] = n >= 2 * K + 1 ? 2 * K + 1 : n;
        span *= g.nofs3[a] * (p->L[a] / n);
        nc *= n;
    }
    g.ncell = (int)nc;
    g.S = g.nofs3[1] * g.nofs3[2];
    // shell sampling: the masks index a cell's culled candidate table, the stencil
    // members within R = r_s + skin of the cell, so within the cell's box grown by R
    // (box + slabs + quarter cylinders + ball); the stencil bounds it too
    double vol = span;
    if (!pool && !p->full_list) {
        double w[3], R = p->r_s + p->skin;
        for (int a = 0; a < 3; ++a) w[a] = p->L[a] / g.n3[a];
        const double grown = w[0] * w[1] * w[2] + 2.0 * R * (w[0] * w[1] + w[1] * w[2] + w[2] * w[0]) +
                             kPi * R * R * (w[0] + w[1] + w[2]) + 4.0 / 3.0 * kPi * R * R * R;
        vol = grown < span ? grown : span;
    }
    int mcap = p->cap_stencil > 0 ? p->cap_stencil : (int)std::ceil(1.3 * rho * vol + 96.0);
    g.mcap = mcap > N ? N : mcap;
    g.core_mean = rho * 4.0 / 3.0 * kPi * std::pow(p->r_c + p->skin, 3);
    g.full_mean = rho * 4.0 / 3.0 * kPi * std::pow(p->r_s + p->skin, 3);
    return g;
}

Plan make_plan(const rbl_params *prm, int R, const int *Ns)
{
    Plan P{};
    P.R = R;
    long long slots = 0, cells = 0, n_real = 0, max_slots = 0;
    int S = 1, mcap = 32;
    double core_mean = 0.0, full_mean = 0.0;
    for (int r = 0; r < R; ++r) {
        Geo g = replica_geo(&prm[r], Ns[r]);
        slots += round_up_ll(Ns[r], kTile);
        if (round_up_ll(Ns[r], kTile) > max_slots) max_slots = round_up_ll(Ns[r], kTile);
        cells += g.ncell + 1;
        n_real += Ns[r];
        S = g.S > S ? g.S : S;
        mcap = g.mcap > mcap ? g.mcap : mcap;
        core_mean = g.core_mean > core_mean ? g.core_mean : core_mean;
        full_mean = g.full_mean > full_mean ? g.full_mean : full_mean;
    }
    const rbl_params *p = &prm[0];
    P.N = (int)slots;
    P.ntile = P.N / kTile;
    P.ncell = (int)cells;
    P.n_real = n_real;
    P.S = S;
    P.Mcap = round_up(mcap, 32);
    // the stencil pool and the full list need no masks; the full list's rows are
    // explicit (row-major) in the core array, cap_c entries each
    P.W = (prm[0].sampling == RBL_SAMPLE_STENCIL || p->full_list) ? 0 : P.Mcap / 32;
    const double row_mean = p->full_list ? full_mean : core_mean;
    P.cap_c = p->cap_core > 0 ? round_up(p->cap_core, p->full_list ? 8 : 1)
                              : round_up((int)std::ceil(1.6 * row_mean + 24.0), 8);
    P.n_scan_blocks = (P.ncell + 2047) / 2048;
    P.pchunks = (int)((max_slots / kMinBlock + kChunkGroups - 1) / kChunkGroups);
    const size_t Nz = (size_t)P.N;
    const size_t Nq = p->potential == RBL_POT_LJ_EWALD ? Nz : 0; // charges only with the Ewald term
    size_t st = 64 * (size_t)n_real + 4096;            // packed x, v and images (host copies, checkpoints)
    if (st < 4 * Nz * (size_t)(p->p + 1)) st = 4 * Nz * (size_t)(p->p + 1); // batch hook
    if (st < sizeof(rbl_obs) * (size_t)R) st = sizeof(rbl_obs) * (size_t)R;   // rbl_obs[R]
    if (st < (1u << 20)) st = 1u << 20;
    P.staging_bytes = st;
    const size_t sizes[] = {
        24 * Nz, 24 * Nz, 24 * Nz, 24 * Nz,         // x, x_alt, v, v_alt
        4 * Nz, 4 * Nz,                             // tag, tag_alt
        16 * Nz, 16 * Nz, 16 * Nz,                  // pos, pos_alt, ubuild
        24 * Nz,                                    // F
        4 * Nz, 4 * Nz,                             // cell, order
        4 * ((size_t)P.ncell + 1), 4 * ((size_t)P.ncell + 1), 4 * ((size_t)P.ncell + 1), // counts, start, fill
        4 * ((size_t)P.n_scan_blocks + 1),          // blocksums
        16 * (size_t)P.ncell * (size_t)P.S,         // seg_tab
        P.W > 0 ? 4 * (size_t)P.ncell * (size_t)P.Mcap : 0, // ctab (shell sampling)
        P.W > 0 ? 4 * (size_t)P.ncell : 0,          // ctab_n
        4 * Nz * (size_t)P.cap_c, 4 * Nz,           // core, n_core
        4 * Nz * (size_t)P.W, 4 * Nz,               // mask, n_shell
        4 * Nz,                                     // hcell
        64 * (Nz / kMinBlock),                      // partials [blocks][8] doubles, any block size >= kMinBlock
        64 * (size_t)R * (size_t)P.pchunks,         // partials2 [R][pchunks][8] doubles
        sizeof(Box) * (size_t)R,                    // box
        8 * (size_t)P.ntile,                        // tile
        4 * (size_t)P.ncell,                        // cell_rep
        sizeof(RepScalars) * (size_t)R,             // rs
        sizeof(DevScalars),                         // sc
        P.staging_bytes,                            // staging
        64 * (size_t)round_up(R, 16),               // kin_acc [8][R rounded up to 16]
        8 * Nq, 4 * Nq, 8 * Nq,                     // q, q32, q_in
    };
    P.n = (int)(sizeof(sizes) / sizeof(sizes[0]));
    size_t o = 0;
    for (int k = 0; k < P.n; ++k) {
        P.off[k] = o;
        o += align256(sizes[k]);
    }
    P.total = o;
    return P;
}

// Replica r's table entry: box, thermostat amplitude, seed, cell grid and stencil.
Box make_box(const rbl_params *p, int N, int first, int c0, int in0)
{
    Box b{};
    Geo g = replica_geo(p, N);
    const int K = p->sampling == RBL_SAMPLE_STENCIL ? (int)std::floor(p->r_s / p->r_c) + 1 : p->cells_per_cutoff;
    for (int a = 0; a < 3; ++a) {
        b.L[a] = p->L[a];
        b.inv[a] = 4294967296.0 / p->L[a];
        b.h[a] = (float)(p->L[a] / 4294967296.0);
        b.n[a] = g.n3[a];
        b.nofs[a] = g.nofs3[a];
        for (int o = 0; o < g.nofs3[a]; ++o) b.ofs[a][o] = g.n3[a] >= 2 * K + 1 ? o - K : o;
    }
    const double c1 = std::exp(-p->gamma * p->dt);
    b.c2f = (float)std::sqrt((1.0 - c1 * c1) * p->T);
    b.T = p->T;
    b.seed = p->seed;
    b.N = N;
    b.first = first;
    b.slots = round_up(N, kTile);
    b.in0 = in0;
    b.c0 = c0;
    b.ncell = g.ncell;
    b.S = g.S;
    // rbl_obs constants (host arithmetic without contraction: each operation rounded once)
    const double n = (double)N, rs = p->r_s;
    b.V = (b.L[0] * b.L[1]) * b.L[2];
    b.n3 = 3.0 * n;
    b.rho = n / b.V;
    b.V3 = 3.0 * b.V;
    const double i3 = 1.0 / ((rs * rs) * rs);
    const double i9 = (i3 * i3) * i3;
    b.U_tail = (((8.0 / 3.0) * kPi) * b.rho) * (i9 / 3.0 - i3);
    b.P_tail = ((((16.0 / 3.0) * kPi) * b.rho) * b.rho) * ((2.0 * i9) / 3.0 - i3);
    return b;
}

// Kernel view over a laid-out workspace (the shared parameters come from prm).
void assign_view(View &v, const rbl_params *prm, const Plan &P, char *base)
{
    v = View{};
    v.N = P.N;
    v.R = P.R;
    v.ntile = P.ntile;
    v.p = prm->p;
    v.K = prm->cells_per_cutoff;
    v.cap_c = P.cap_c;
    v.W = P.W;
    v.S = P.S;
    v.Mcap = P.Mcap;
    v.full_list = prm->full_list ? 1 : 0;
    v.precision = prm->precision;
    v.subtract = prm->subtract_net_force ? 1 : 0;
    v.sampling = prm->sampling;
    v.potential = prm->potential;
    v.alpha = prm->alpha;
    v.ka = 2.0 * prm->alpha / std::sqrt(kPi);
    v.alpha32 = (float)v.alpha;
    v.ka32 = (float)v.ka;
    // the force kernel's fastest block before any autotuning: 256 threads for FP32
    // shell sampling and the full list, 128 otherwise (measured at N = 2^20)
    v.force_threads = (prm->precision == RBL_FP32 && !prm->sampling) ? 256 : 128;
    v.build_warps = 4;
    v.ncell = P.ncell;
    const double rc = prm->r_c, rs = prm->r_s, sk = prm->skin;
    const double lo = rc - sk > 0.0 ? rc - sk : 0.0;
    v.t_core_list = (float)((rc + sk) * (rc + sk));
    v.t_shell_lo = (float)(lo * lo);
    v.t_cut_list = (float)((rs + sk) * (rs + sk));
    v.t_cull = (float)((rs + sk) * (rs + sk) * (1.0 + 1.0 / 4096.0));
    v.t_rc2 = (float)(rc * rc);
    v.t_rs2 = (float)(rs * rs);
    v.t_disp = (float)(0.25 * sk * sk);
    v.dt = prm->dt;
    v.gamma = prm->gamma;
    v.c1 = std::exp(-prm->gamma * prm->dt);
    int k = 0;
    v.x = (double *)(base + P.off[k++]);
    v.x_alt = (double *)(base + P.off[k++]);
    v.v = (double *)(base + P.off[k++]);
    v.v_alt = (double *)(base + P.off[k++]);
    v.tag = (int *)(base + P.off[k++]);
    v.tag_alt = (int *)(base + P.off[k++]);
    v.pos = (int4 *)(base + P.off[k++]);
    v.pos_alt = (int4 *)(base + P.off[k++]);
    v.ubuild = (int4 *)(base + P.off[k++]);
    v.F = (void *)(base + P.off[k++]);
    v.cell = (int *)(base + P.off[k++]);
    v.order = (int *)(base + P.off[k++]);
    v.counts = (int *)(base + P.off[k++]);
    v.start = (int *)(base + P.off[k++]);
    v.fill = (int *)(base + P.off[k++]);
    v.blocksums = (int *)(base + P.off[k++]);
    v.seg_tab = (int4 *)(base + P.off[k++]);
    v.ctab = (int *)(base + P.off[k++]);
    v.ctab_n = (int *)(base + P.off[k++]);
    v.core = (int *)(base + P.off[k++]);
    v.n_core = (int *)(base + P.off[k++]);
    v.mask = (unsigned *)(base + P.off[k++]);
    v.n_shell = (int *)(base + P.off[k++]);
    v.hcell = (int *)(base + P.off[k++]);
    v.partials = (double *)(base + P.off[k++]);
    v.partials2 = (double *)(base + P.off[k++]);
    v.pchunks = P.pchunks;
    v.box = (const Box *)(base + P.off[k++]);
    v.tile = (const int2 *)(base + P.off[k++]);
    v.cell_rep = (const int *)(base + P.off[k++]);
    v.rs = (RepScalars *)(base + P.off[k++]);
    v.sc = (DevScalars *)(base + P.off[k++]);
    v.staging = (double *)(base + P.off[k++]);
    v.kin_acc = (unsigned long long *)(base + P.off[k++]);
    v.kin_stride = round_up(P.R, 16);
    if (prm->potential == RBL_POT_LJ_EWALD) {
        v.q = (double *)(base + P.off[k++]);
        v.q32 = (float *)(base + P.off[k++]);
        v.q_in = (double *)(base + P.off[k++]);
    }
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_err(ctx, "%s failed: %s", #call, cudaGetErrorString(e_));                \
            return RBL_ECUDA;                                                            \
        }                                                                                \
    } while (0)

rbl_status read_scalars(rbl_ctx *ctx, bool replicas = false)
{
    CK(cudaMemcpyAsync(ctx->h_sc, ctx->view.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, ctx->stream));
    if (replicas)
        CK(cudaMemcpyAsync(ctx->h_rs, ctx->view.rs, sizeof(RepScalars) * (size_t)ctx->R, cudaMemcpyDeviceToHost,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RBL_OK;
}

rbl_status check_flags(rbl_ctx *ctx, bool replicas = false)
{
    rbl_status st = read_scalars(ctx, replicas);
    if (st != RBL_OK) return st;
    unsigned f = ctx->h_sc->flags;
    // a blow-up first: row or cell overflows can follow from it
    if (f & kFlagNonFinite) {
        set_err(ctx, "non-finite position, velocity or force, a force beyond the fixed-point range (overlapping "
                     "particles), or a particle that moved more than a box length in one step");
        return RBL_ENONFINITE;
    }
    if (f & (kFlagOverflow | kFlagCellOverflow)) {
        if (!replicas) read_scalars(ctx, true);
        int nc = 0, m = 0;
        for (int r = 0; r < ctx->R; ++r) {
            nc = ctx->h_rs[r].nc_max > nc ? ctx->h_rs[r].nc_max : nc;
            m = ctx->h_rs[r].t_max > m ? ctx->h_rs[r].t_max : m;
        }
        set_err(ctx, "capacity exceeded (longest core row %d / cap %d, largest candidate table %d / cap %d)", nc,
                ctx->view.cap_c, m, ctx->view.Mcap);
        return RBL_EOVERFLOW;
    }
    if (f & kFlagRngLimit) {
        set_err(ctx, "bounded-draw rejection limit reached");
        return RBL_ETIMEOUT;
    }
    return RBL_OK;
}

rbl_status ensure_lists(rbl_ctx *ctx)
{
    if (ctx->lists_valid) return RBL_OK;
    if (ctx->phase_timing) {
        // a rebuild outside the step loop, timed on its own: the sort chain and the list
        // build, with none of the skipped launches of the steps that do not rebuild
        for (int k = 0; k < 3; ++k)
            if (!ctx->rb_ev[k]) CK(cudaEventCreate(&ctx->rb_ev[k]));
        CK(cudaEventRecord(ctx->rb_ev[0], ctx->stream));
        CK(launch_rebuild_sort(ctx->view, ctx->n_scan_blocks, false, ctx->stream));
        CK(cudaEventRecord(ctx->rb_ev[1], ctx->stream));
        CK(launch_rebuild_lists(ctx->view, false, ctx->stream));
        CK(cudaEventRecord(ctx->rb_ev[2], ctx->stream));
        CK(cudaEventSynchronize(ctx->rb_ev[2]));
        for (int k = 0; k < 2; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->rb_ev[k], ctx->rb_ev[k + 1]));
            ctx->rebuild_ms[k] += ms;
        }
        ctx->rebuild_n += 1;
    } else {
        CK(launch_rebuild(ctx->view, ctx->n_scan_blocks, false, ctx->stream));
    }
    ctx->lists_valid = 1;
    ctx->force_valid = 0;
    return RBL_OK;
}

rbl_status ensure_force(rbl_ctx *ctx, bool energy)
{
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    if (ctx->force_valid && (!energy || ctx->energy_valid)) return RBL_OK;
    CK(launch_forces(ctx->view, 0, 0, energy, ctx->stream));
    ctx->force_valid = 1;
    ctx->energy_valid = energy || ctx->view.precision == RBL_FP64;
    return RBL_OK;
}

// Applies the half kick a step call left pending (before anything that changes the
// force it is due with: charges, a forced rebuild).
rbl_status resolve_kick(rbl_ctx *ctx)
{
    if (!ctx->kick_pending) return RBL_OK;
    rbl_status st = ensure_force(ctx, false);
    if (st != RBL_OK) return st;
    CK(launch_integrate(ctx->view, 0.5 * ctx->prm.dt, false, ctx->stream));
    ctx->kick_pending = 0;
    return RBL_OK;
}

// Phases of a timed step: kick/drift/thermostat, cell sort chain, list build,
// force kernel, force reduction.
constexpr int kPhases = 5, kPhaseEvents = kPhases + 1;

// One steady-state step: kick(ck)+drift+O, conditional rebuild, force at n+1.
// ev (optional): kPhaseEvents events recorded at the phase boundaries.
cudaError_t enqueue_step(rbl_ctx *ctx, double ck, bool energy, cudaEvent_t *ev = nullptr)
{
    cudaError_t e = cudaSuccess;
    if (ev) e = cudaEventRecord(ev[0], ctx->stream);
    if (e == cudaSuccess) e = launch_integrate(ctx->view, ck, true, ctx->stream);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], ctx->stream);
    if (e == cudaSuccess) e = launch_rebuild_sort(ctx->view, ctx->n_scan_blocks, true, ctx->stream);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], ctx->stream);
    if (e == cudaSuccess) e = launch_rebuild_lists(ctx->view, true, ctx->stream);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], ctx->stream);
    if (e == cudaSuccess) e = launch_force_kernel(ctx->view, 1, energy, ctx->stream);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[4], ctx->stream);
    if (e == cudaSuccess) e = launch_force_finish(ctx->view, 1, energy, ctx->stream);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[5], ctx->stream);
    return e;
}

rbl_status ensure_events(rbl_ctx *ctx, int steps)
{
    if (ctx->ev_cap >= steps) return RBL_OK;
    int cap = steps < 64 ? 64 : steps;
    cudaEvent_t *ev = (cudaEvent_t *)std::calloc((size_t)cap * kPhaseEvents, sizeof(cudaEvent_t));
    if (!ev) return RBL_ENOMEM;
    for (int k = 0; k < ctx->ev_cap * kPhaseEvents; ++k) ev[k] = ctx->ev[k];
    for (int k = ctx->ev_cap * kPhaseEvents; k < cap * kPhaseEvents; ++k) CK(cudaEventCreate(&ev[k]));
    std::free(ctx->ev);
    ctx->ev = ev;
    ctx->ev_cap = cap;
    return RBL_OK;
}

// Steady-state step as a CUDA graph: kick/drift/thermostat, a kernel that copies the
// device rebuild flag into a conditional handle, an IF node whose body is the whole
// rebuild chain, then the force and its reduction.  No host round trip and no
// empty launches when no rebuild is due.
// The captured steps.  Every step is kick(ck) + drift (+ O), the device-conditional
// rebuild chain, the force at n + 1 and its reduction.  A call's last step ends
// after its force (with the energy estimates refreshed); its closing half kick is
// left pending and applied by the next call's first step together with that step's
// opening half kick, one kick of dt as between the steps inside a call, so the
// trajectory does not depend on how a run is split into calls.  Only the first step
// after a new state (nothing pending) opens with a half kick.
enum StepGraph { kGraphMid = 0, kGraphFirst = 1, kGraphMidE = 2, kGraphFirstE = 3 };

rbl_status ensure_graph(rbl_ctx *ctx, int kind)
{
    if (ctx->graph_exec[kind]) return RBL_OK;
    const bool half = kind == kGraphFirst || kind == kGraphFirstE;
    const bool last = kind == kGraphMidE || kind == kGraphFirstE;
    const double ck = half ? 0.5 * ctx->prm.dt : ctx->prm.dt;
    cudaStream_t s = ctx->stream;
    CK(launch_force_kernel(ctx->view, 1, last, s, true)); // kernel attributes, before the capture
    cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle handle;
    cudaError_t e = cudaGraphConditionalHandleCreate(&handle, g, 0, cudaGraphCondAssignDefault);
    cudaGraphNode_t cond_node = nullptr;
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, mode);
    if (e == cudaSuccess) {
        cudaError_t ec = launch_integrate(ctx->view, ck, true, s);
        if (ec == cudaSuccess) ec = launch_set_rebuild_condition(ctx->view, handle, s);
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        if (ec == cudaSuccess) ec = cudaStreamGetCaptureInfo(s, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (ec == cudaSuccess) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            ec = cudaGraphAddNode(&cond_node, g, deps, nullptr, ndeps, &cp);
        }
        if (ec == cudaSuccess)
            ec = cudaStreamUpdateCaptureDependencies(s, &cond_node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (ec == cudaSuccess) ec = launch_forces(ctx->view, 1, 1, last, s);
        cudaGraph_t gout = nullptr;
        e = cudaStreamEndCapture(s, &gout);
        if (ec != cudaSuccess) e = ec;
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, mode);
        if (e == cudaSuccess) {
            // conditional kernels: inside the IF body some replica is due, and each
            // kernel still skips the replicas whose own flag is down
            cudaError_t ec = launch_rebuild(ctx->view, ctx->n_scan_blocks, true, s);
            cudaGraph_t bout = nullptr;
            e = cudaStreamEndCapture(s, &bout);
            if (ec != cudaSuccess) e = ec;
        }
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_err(ctx, "building the step graph failed: %s", cudaGetErrorString(e));
        return RBL_ECUDA;
    }
    ctx->graph_exec[kind] = ex;
    return RBL_OK;
}

void drop_graphs(rbl_ctx *ctx)
{
    for (cudaGraphExec_t &g : ctx->graph_exec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

rbl_status create_impl(const rbl_params *prm, int R, const int *Ns, void *workspace, size_t workspace_bytes,
                       void *stream, rbl_ctx **out)
{
    if (!out) return RBL_EINVAL;
    *out = nullptr;
    rbl_ctx *ctx = new (std::nothrow) rbl_ctx();
    if (!ctx) return RBL_ENOMEM;
    rbl_status st = validate_batch(prm, R, Ns, ctx->err, sizeof(ctx->err));
    if (st != RBL_OK) {
        // keep the handle so the caller can read the message; it holds no device state
        *out = ctx;
        return st;
    }
    const Plan P = make_plan(prm, R, Ns);
    if (!workspace || workspace_bytes < P.total || ((uintptr_t)workspace & 255u)) {
        set_err(ctx, "workspace must be 256-byte aligned and at least %zu bytes (got %zu)", P.total,
                workspace_bytes);
        *out = ctx;
        return workspace_bytes < P.total ? RBL_ENOMEM : RBL_EINVAL;
    }
    ctx->prm = prm[0];
    ctx->stream = (cudaStream_t)stream;
    ctx->R = R;
    ctx->n_real = P.n_real;
    ctx->n_scan_blocks = P.n_scan_blocks;
    ctx->step = 0;
    ctx->staging_bytes = P.staging_bytes;
    ctx->h_sc = new (std::nothrow) DevScalars();
    ctx->h_rs = new (std::nothrow) RepScalars[R]();
    ctx->h_box = new (std::nothrow) Box[R]();
    ctx->h_tile = new (std::nothrow) int2[P.ntile]();
    ctx->h_cell_rep = new (std::nothrow) int[P.ncell]();
    if (!ctx->h_sc || !ctx->h_rs || !ctx->h_box || !ctx->h_tile || !ctx->h_cell_rep) {
        set_err(ctx, "host tables: out of memory");
        *out = ctx;
        return RBL_ENOMEM;
    }
    // replica table: replicas in order, each on whole tiles and followed by its pad cell
    int first = 0, c0 = 0, in0 = 0;
    for (int r = 0; r < R; ++r) {
        Box &b = ctx->h_box[r];
        b = make_box(&prm[r], Ns[r], first, c0, in0);
        for (int t = first / kTile; t < (first + b.slots) / kTile; ++t) ctx->h_tile[t] = make_int2(r, first + b.N);
        for (int c = c0; c <= c0 + b.ncell; ++c) ctx->h_cell_rep[c] = r;
        first += b.slots;
        c0 += b.ncell + 1;
        in0 += b.N;
    }
    View &v = ctx->view;
    assign_view(v, &prm[0], P, (char *)workspace);
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync((void *)v.box, ctx->h_box, sizeof(Box) * (size_t)R, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)v.tile, ctx->h_tile, 8 * (size_t)P.ntile, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)v.cell_rep, ctx->h_cell_rep, 4 * (size_t)P.ncell, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.sc, 0, sizeof(DevScalars), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.rs, 0, sizeof(RepScalars) * (size_t)R, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.kin_acc, 0, 64 * (size_t)v.kin_stride, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.F, 0, 24 * (size_t)P.N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.partials, 0, 64 * ((size_t)P.N / kMinBlock), s);
    if (e == cudaSuccess && v.q) {
        e = cudaMemsetAsync(v.q, 0, 8 * (size_t)P.N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(v.q32, 0, 4 * (size_t)P.N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(v.q_in, 0, 8 * (size_t)P.N, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_err(ctx, "initialisation failed: %s", cudaGetErrorString(e));
        *out = ctx;
        return RBL_ECUDA;
    }
    *out = ctx;
    return RBL_OK;
}

} // namespace

extern "C" {

void rbl_params_default(rbl_params *prm)
{
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->p = 10;
    prm->dt = 0.005;
    prm->T = 1.0;
    prm->seed = 1;
    prm->precision = RBL_FP32;
    prm->subtract_net_force = 1;
    prm->cells_per_cutoff = 2;
}

rbl_status rbl_workspace_size(const rbl_params *prm, int N, size_t *bytes)
{
    return rbl_workspace_size_batch(prm, 1, &N, bytes);
}

rbl_status rbl_workspace_size_batch(const rbl_params *prm, int R, const int *N, size_t *bytes)
{
    if (!bytes) return RBL_EINVAL;
    rbl_status st = validate_batch(prm, R, N, nullptr, 0);
    if (st != RBL_OK) return st;
    *bytes = make_plan(prm, R, N).total;
    return RBL_OK;
}

rbl_status rbl_create(const rbl_params *prm, int N, void *workspace, size_t workspace_bytes, void *stream,
                      rbl_ctx **out)
{
    return create_impl(prm, 1, &N, workspace, workspace_bytes, stream, out);
}

rbl_status rbl_create_batch(const rbl_params *prm, int R, const int *N, void *workspace, size_t workspace_bytes,
                            void *stream, rbl_ctx **out)
{
    return create_impl(prm, R, N, workspace, workspace_bytes, stream, out);
}

int rbl_replicas(const rbl_ctx *ctx) { return ctx ? ctx->R : 0; }

// Device address of page-locked host memory mapped into the device's address space
// (kernels then read or write it over the CPU-GPU link directly, with no staging
// copy), or nullptr for any other host memory.
static void *mapped_alias(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
        return at.devicePointer;
    cudaGetLastError(); // an unregistered pointer is not an error here
    return nullptr;
}

rbl_status rbl_set_state(rbl_ctx *ctx, const double *x, const double *v, long long step, int ptr_is_device)
{
    if (!ctx || !x || step < 0) return RBL_EINVAL;
    size_t bytes = 24 * (size_t)ctx->n_real;
    const double *dx = x, *dv = v;
    if (!ptr_is_device) {
        // page-locked buffers are read by the load kernel itself; others through the
        // staging area (the call waits for the kernel either way)
        double *sx = ctx->view.staging, *sv = ctx->view.staging + 3 * (size_t)ctx->n_real;
        dx = (const double *)mapped_alias(x);
        if (!dx) {
            CK(cudaMemcpyAsync(sx, x, bytes, cudaMemcpyHostToDevice, ctx->stream));
            dx = sx;
        }
        dv = v ? (const double *)mapped_alias(v) : nullptr;
        if (v && !dv) {
            CK(cudaMemcpyAsync(sv, v, bytes, cudaMemcpyHostToDevice, ctx->stream));
            dv = sv;
        }
    }
    DevScalars z{};
    *ctx->h_sc = z;
    ctx->h_sc->step = (unsigned long long)step;
    CK(cudaMemcpyAsync(ctx->view.sc, ctx->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->view.rs, 0, sizeof(RepScalars) * (size_t)ctx->R, ctx->stream));
    CK(launch_load_state(ctx->view, dx, dv, ctx->stream));
    ctx->step = step;
    ctx->lists_valid = 0;
    ctx->force_valid = 0;
    ctx->energy_valid = 0;
    ctx->kick_pending = 0;
    if (!ptr_is_device) {
        rbl_status st = check_flags(ctx);
        if (st != RBL_OK) return st;
    }
    return RBL_OK;
}

rbl_status rbl_set_charges(rbl_ctx *ctx, const double *q)
{
    if (!ctx || !q) return RBL_EINVAL;
    if (!ctx->view.q) {
        set_err(ctx, "rbl_set_charges needs potential RBL_POT_LJ_EWALD");
        return RBL_EINVAL;
    }
    for (long long k = 0; k < ctx->n_real; ++k)
        if (!std::isfinite(q[k])) {
            set_err(ctx, "charge %lld is not finite", k);
            return RBL_EINVAL;
        }
    rbl_status st = resolve_kick(ctx); // the pending half kick is due with the old charges' force
    if (st != RBL_OK) return st;
    double *sq = ctx->view.staging;
    CK(cudaMemcpyAsync(sq, q, 8 * (size_t)ctx->n_real, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_set_charges(ctx->view, sq, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->force_valid = 0;
    ctx->energy_valid = 0;
    return RBL_OK;
}

rbl_status rbl_get_state(rbl_ctx *ctx, double *x, double *v, long long *step, int ptr_is_device)
{
    if (!ctx) return RBL_EINVAL;
    if (step) *step = ctx->step;
    if (!x && !v) return RBL_OK;
    size_t bytes = 24 * (size_t)ctx->n_real;
    // velocities as of the end of the last step: with its closing half kick
    const double ck = ctx->kick_pending ? 0.5 * ctx->prm.dt : 0.0;
    if (ptr_is_device) {
        CK(launch_store_state(ctx->view, x, v, ctx->stream, ck));
        return RBL_OK;
    }
    // through the staging area whatever the host memory: the store kernel writes in tag
    // order from cell order, scattered writes that cost 3x more over the CPU-GPU link
    // than a bulk copy after them (measured: 0.98 against 0.31 ms for 2^20 particles)
    double *sx = ctx->view.staging, *sv = ctx->view.staging + 3 * (size_t)ctx->n_real;
    CK(launch_store_state(ctx->view, x ? sx : nullptr, v ? sv : nullptr, ctx->stream, ck));
    if (x) CK(cudaMemcpyAsync(x, sx, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    if (v) CK(cudaMemcpyAsync(v, sv, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RBL_OK;
}

// Checkpoint buffer: header | n_rebuild[R] | x[n][3] | v[n][3] (doubles) | images[n][3]
// (uint32), n = every replica's particles, tag order packed over replicas.
struct CkptHeader {
    char magic[8];          // "RBLCKPT1"
    long long n_real;
    long long step;
    int R;
    int precision;
    int lists_valid;        // the lists were built from the saved images
    int kick_pending;       // the velocities still lack the last step's closing half kick
    int reserved[2];
};

static size_t ckpt_head_bytes(int R) { return (sizeof(CkptHeader) + 8 * (size_t)R + 15) & ~(size_t)15; }

rbl_status rbl_checkpoint_size(const rbl_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return RBL_EINVAL;
    *bytes = ckpt_head_bytes(ctx->R) + 60 * (size_t)ctx->n_real;
    return RBL_OK;
}

rbl_status rbl_save_checkpoint(rbl_ctx *ctx, void *buf, int ptr_is_device)
{
    if (!ctx || !buf) return RBL_EINVAL;
    rbl_status st = read_scalars(ctx, true);
    if (st != RBL_OK) return st;
    const size_t head = ckpt_head_bytes(ctx->R), n = (size_t)ctx->n_real;
    std::vector<char> h(head, 0);
    CkptHeader hd{};
    std::memcpy(hd.magic, "RBLCKPT1", 8);
    hd.n_real = ctx->n_real;
    hd.step = ctx->step;
    hd.R = ctx->R;
    hd.precision = ctx->prm.precision;
    hd.lists_valid = ctx->lists_valid;
    hd.kick_pending = ctx->kick_pending;
    std::memcpy(h.data(), &hd, sizeof(hd));
    for (int r = 0; r < ctx->R; ++r)
        std::memcpy(h.data() + sizeof(CkptHeader) + 8 * (size_t)r, &ctx->h_rs[r].n_rebuild, 8);
    char *dst = ptr_is_device ? (char *)buf : (char *)ctx->view.staging;
    double *x = (double *)(dst + head);
    unsigned *img = (unsigned *)(x + 6 * n);
    CK(launch_store_state(ctx->view, x, x + 3 * n, ctx->stream));
    CK(launch_store_images(ctx->view, img, ctx->stream));
    if (ptr_is_device) {
        CK(cudaMemcpyAsync(buf, h.data(), head, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return RBL_OK;
    }
    std::memcpy(buf, h.data(), head);
    CK(cudaMemcpyAsync((char *)buf + head, dst + head, 60 * n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RBL_OK;
}

rbl_status rbl_load_checkpoint(rbl_ctx *ctx, const void *buf, int ptr_is_device)
{
    if (!ctx || !buf) return RBL_EINVAL;
    const size_t head = ckpt_head_bytes(ctx->R), n = (size_t)ctx->n_real;
    std::vector<char> h(head, 0);
    if (ptr_is_device) {
        CK(cudaMemcpyAsync(h.data(), buf, head, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    } else {
        std::memcpy(h.data(), buf, head);
    }
    CkptHeader hd;
    std::memcpy(&hd, h.data(), sizeof(hd));
    if (std::memcmp(hd.magic, "RBLCKPT1", 8) != 0) {
        set_err(ctx, "not an rbl checkpoint");
        return RBL_EINVAL;
    }
    if (hd.n_real != ctx->n_real || hd.R != ctx->R || hd.precision != ctx->prm.precision || hd.step < 0) {
        set_err(ctx, "checkpoint of %lld particles in %d replicas (precision %d) does not fit this context (%lld in %d, %d)",
                hd.n_real, hd.R, hd.precision, ctx->n_real, ctx->R, ctx->prm.precision);
        return RBL_EINVAL;
    }
    const char *src = (const char *)buf;
    if (!ptr_is_device) {
        CK(cudaMemcpyAsync(ctx->view.staging, src + head, 60 * n, cudaMemcpyHostToDevice, ctx->stream));
        src = (const char *)ctx->view.staging - head;
    }
    const double *x = (const double *)(src + head);
    const unsigned *img = (const unsigned *)(x + 6 * n);
    DevScalars z{};
    *ctx->h_sc = z;
    ctx->h_sc->step = (unsigned long long)hd.step;
    CK(cudaMemcpyAsync(ctx->view.sc, ctx->h_sc, sizeof(DevScalars), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->view.rs, 0, sizeof(RepScalars) * (size_t)ctx->R, ctx->stream));
    CK(launch_load_state(ctx->view, x, x + 3 * n, ctx->stream));
    CK(launch_load_images(ctx->view, img, ctx->stream));
    if (hd.lists_valid) {
        // the lists of the saved context: the rebuild chain run on the saved build
        // images (in place of the current ones) puts the particles in that build's
        // cell order and rebuilds its rows; then the current images are recomputed
        // from the (permuted) positions
        View vb = ctx->view;
        vb.pos = vb.ubuild;
        CK(launch_rebuild(vb, ctx->n_scan_blocks, false, ctx->stream));
        CK(launch_requantize(ctx->view, ctx->stream));
    }
    rbl_status st = read_scalars(ctx, true);
    if (st != RBL_OK) return st;
    for (int r = 0; r < ctx->R; ++r)
        std::memcpy(&ctx->h_rs[r].n_rebuild, h.data() + sizeof(CkptHeader) + 8 * (size_t)r, 8);
    CK(cudaMemcpyAsync(ctx->view.rs, ctx->h_rs, sizeof(RepScalars) * (size_t)ctx->R, cudaMemcpyHostToDevice,
                       ctx->stream));
    ctx->step = hd.step;
    ctx->lists_valid = hd.lists_valid ? 1 : 0;
    ctx->force_valid = 0;
    ctx->energy_valid = 0;
    ctx->kick_pending = hd.kick_pending ? 1 : 0; // the force it is due with is recomputed first
    return check_flags(ctx);
}

rbl_status rbl_build_lists(rbl_ctx *ctx)
{
    if (!ctx) return RBL_EINVAL;
    rbl_status st0 = resolve_kick(ctx); // due with the force of the current lists
    if (st0 != RBL_OK) return st0;
    ctx->lists_valid = 0;
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    return check_flags(ctx);
}

rbl_status rbl_forces(rbl_ctx *ctx, double *F_out, int ptr_is_device)
{
    if (!ctx) return RBL_EINVAL;
    ctx->force_valid = 0;
    rbl_status st = ensure_force(ctx, true);
    if (st != RBL_OK) return st;
    if (F_out) {
        if (ptr_is_device) {
            CK(launch_store_forces(ctx->view, F_out, ctx->stream));
        } else {
            CK(launch_store_forces(ctx->view, ctx->view.staging, ctx->stream));
            CK(cudaMemcpyAsync(F_out, ctx->view.staging, 24 * (size_t)ctx->n_real, cudaMemcpyDeviceToHost,
                               ctx->stream));
            return check_flags(ctx);
        }
    }
    return RBL_OK;
}

// n steps; sync: wait for them and report the device flags.
static rbl_status step_impl(rbl_ctx *ctx, int n, bool sync)
{
    if (!ctx || n < 0) return RBL_EINVAL;
    if (n == 0) return RBL_OK;
    rbl_status st = ensure_force(ctx, false);
    if (st != RBL_OK) return st;
    // every step kicks by dt (the previous step's closing half kick and its own
    // opening one), except the first step after a new state, which opens with a half
    // kick; the last step also refreshes the energy/virial estimates and leaves its
    // closing half kick pending
    const double dt = ctx->prm.dt, ck0 = ctx->kick_pending ? dt : 0.5 * dt;
    if (ctx->phase_timing) {
        st = ensure_events(ctx, n);
        if (st != RBL_OK) return st;
        for (int k = 0; k < n; ++k) CK(enqueue_step(ctx, k == 0 ? ck0 : dt, k == n - 1, ctx->ev + kPhaseEvents * k));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int k = 0; k < n; ++k)
            for (int ph = 0; ph < kPhases; ++ph) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ctx->ev[kPhaseEvents * k + ph], ctx->ev[kPhaseEvents * k + ph + 1]));
                ctx->phase_ms[ph] += ms;
            }
        ctx->phase_steps += n;
        ctx->step += n;
        ctx->force_valid = 1;
        ctx->energy_valid = 1;
        ctx->kick_pending = 1;
        return check_flags(ctx);
    }
    if (ctx->stream == nullptr) {
        // the legacy default stream cannot be captured: launch directly
        for (int k = 0; k < n; ++k) CK(enqueue_step(ctx, k == 0 ? ck0 : dt, k == n - 1));
    } else {
        const bool p = ctx->kick_pending != 0;
        const int first = n == 1 ? (p ? kGraphMidE : kGraphFirstE) : (p ? kGraphMid : kGraphFirst);
        st = ensure_graph(ctx, first);
        if (st == RBL_OK && n > 2) st = ensure_graph(ctx, kGraphMid);
        if (st == RBL_OK && n > 1) st = ensure_graph(ctx, kGraphMidE);
        if (st != RBL_OK) return st;
        CK(cudaGraphLaunch(ctx->graph_exec[first], ctx->stream));
        for (int k = 1; k < n - 1; ++k) CK(cudaGraphLaunch(ctx->graph_exec[kGraphMid], ctx->stream));
        if (n > 1) CK(cudaGraphLaunch(ctx->graph_exec[kGraphMidE], ctx->stream));
    }
    ctx->step += n;
    ctx->force_valid = 1;
    ctx->energy_valid = 1;
    ctx->kick_pending = 1;
    return sync ? check_flags(ctx) : RBL_OK;
}


rbl_status rbl_step(rbl_ctx *ctx, int n) { return step_impl(ctx, n, true); }

rbl_status rbl_step_async(rbl_ctx *ctx, int n)
{
    if (ctx && ctx->phase_timing) return step_impl(ctx, n, true); // timed steps wait for their events
    return step_impl(ctx, n, false);
}


// Enqueues the observables launch (kinetic sums and the device-side assembly of
// rbl_obs[R]) and, where out is not written by the kernel itself, its copy to out.
rbl_status enqueue_observables(rbl_ctx *ctx, rbl_obs *out, int ptr_is_device)
{
    rbl_status st = ensure_force(ctx, true);
    if (st != RBL_OK) return st;
    const double ck = ctx->kick_pending ? 0.5 * ctx->prm.dt : 0.0;
    // page-locked host memory (mapped into the device's address space) and device
    // memory are written by the kernel itself; anything else through the staging area
    void *direct = ptr_is_device ? (void *)out : mapped_alias(out);
    if (direct) {
        CK(launch_observables(ctx->view, (rbl_obs *)direct, ck, ctx->stream));
        return RBL_OK;
    }
    rbl_obs *dev = (rbl_obs *)ctx->view.staging;
    CK(launch_observables(ctx->view, dev, ck, ctx->stream));
    CK(cudaMemcpyAsync(out, dev, sizeof(rbl_obs) * (size_t)ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    return RBL_OK;
}

rbl_status rbl_observables(rbl_ctx *ctx, rbl_obs *out)
{
    if (!ctx || !out) return RBL_EINVAL;
    rbl_status st = enqueue_observables(ctx, out, 0);
    if (st != RBL_OK) return st;
    return check_flags(ctx, true);
}

rbl_status rbl_observables_async(rbl_ctx *ctx, rbl_obs *out, int ptr_is_device)
{
    if (!ctx || !out) return RBL_EINVAL;
    return enqueue_observables(ctx, out, ptr_is_device);
}

rbl_status rbl_exact_energy(rbl_ctx *ctx, double *U, double *W)
{
    if (!ctx || !U || !W) return RBL_EINVAL;
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    CK(launch_exact_energy(ctx->view, ctx->stream));
    st = check_flags(ctx, true);
    if (st != RBL_OK) return st;
    for (int r = 0; r < ctx->R; ++r) {
        U[r] = ctx->h_rs[r].u_exact;
        W[r] = ctx->h_rs[r].w_exact;
    }
    return RBL_OK;
}

rbl_status rbl_get_lists(rbl_ctx *ctx, int kind, int *rows, int cap, int *counts)
{
    if (!ctx || !rows || !counts || (kind != 0 && kind != 1) || cap < 1) return RBL_EINVAL;
    if (kind == 0 && ctx->view.full_list) return RBL_EINVAL;
    if (kind == 1 && ctx->view.sampling) {
        set_err(ctx, "stencil-pool sampling builds no shell rows");
        return RBL_EINVAL;
    }
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    st = check_flags(ctx);
    if (st != RBL_OK) return st;
    const View &v = ctx->view;
    const size_t N = (size_t)v.N;
    std::vector<int> tag(N), cnt(N);
    CK(cudaMemcpy(tag.data(), v.tag, 4 * N, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt.data(), kind == 0 ? v.n_core : v.n_shell, 4 * N, cudaMemcpyDeviceToHost));
    // packed row of slot i, or -1 for a padding slot
    std::vector<long long> row_of(N);
    for (size_t i = 0; i < N; ++i) {
        const int2 t = ctx->h_tile[i >> kTileShift];
        row_of[i] = (long long)i < t.y ? (long long)ctx->h_box[t.x].in0 + tag[i] : -1;
        if (row_of[i] >= 0 && cnt[i] > cap) {
            set_err(ctx, "row %lld has %d entries, more than cap %d", row_of[i], cnt[i], cap);
            return RBL_EOVERFLOW;
        }
    }
    if (kind == 0 || v.full_list) {
        // explicit rows: core[k][N] (column-major), or the full list's rows core[N][cap_c]
        std::vector<int> core(N * (size_t)v.cap_c);
        CK(cudaMemcpy(core.data(), v.core, core.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < N; ++i) {
            if (row_of[i] < 0) continue;
            const size_t t = (size_t)row_of[i];
            counts[t] = cnt[i];
            const int n = cnt[i] < v.cap_c ? cnt[i] : v.cap_c;
            for (int k = 0; k < n; ++k)
                rows[t * cap + k] = tag[v.full_list ? core[i * (size_t)v.cap_c + k] : core[(size_t)k * N + i]];
        }
        return RBL_OK;
    }
    // decode the masks on the host: bit b of word w is entry 32 w + b of the home
    // cell's culled candidate table
    std::vector<unsigned> mask(N * (size_t)v.W);
    std::vector<int> ctab(v.W > 0 ? (size_t)v.ncell * v.Mcap : 0);
    std::vector<int> hcell(N);
    if (v.W > 0) {
        CK(cudaMemcpy(mask.data(), v.mask, mask.size() * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ctab.data(), v.ctab, ctab.size() * 4, cudaMemcpyDeviceToHost));
    }
    CK(cudaMemcpy(hcell.data(), v.hcell, 4 * N, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < N; ++i) {
        if (row_of[i] < 0) continue;
        const size_t t = (size_t)row_of[i];
        counts[t] = cnt[i];
        const int *crow = ctab.data() + (size_t)hcell[i] * v.Mcap;
        int k = 0;
        for (int w = 0; w < v.W && k < cnt[i]; ++w) {
            unsigned word = mask[(size_t)w * N + i];
            while (word) {
                int bit = __builtin_ctz(word);
                word &= word - 1u;
                rows[t * cap + k++] = tag[crow[(w << 5) + bit]];
            }
        }
    }
    return RBL_OK;
}

rbl_status rbl_get_rows(rbl_ctx *ctx, int kind, const long long *which, int m, int *rows, int cap, int *counts)
{
    if (!ctx || !which || !rows || !counts || (kind != 0 && kind != 1) || m < 0 || cap < 1) return RBL_EINVAL;
    if (kind == 0 && ctx->view.full_list) return RBL_EINVAL;
    if (kind == 1 && ctx->view.sampling) {
        set_err(ctx, "stencil-pool sampling builds no shell rows");
        return RBL_EINVAL;
    }
    for (int k = 0; k < m; ++k)
        if (which[k] < 0 || which[k] >= ctx->n_real) {
            set_err(ctx, "row %lld out of range", which[k]);
            return RBL_EINVAL;
        }
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    st = check_flags(ctx);
    if (st != RBL_OK) return st;
    const View &v = ctx->view;
    const size_t N = (size_t)v.N;
    std::vector<int> tag(N);
    CK(cudaMemcpy(tag.data(), v.tag, 4 * N, cudaMemcpyDeviceToHost));
    // slot of every requested packed row
    std::vector<long long> slot_of((size_t)ctx->n_real, -1);
    for (size_t i = 0; i < N; ++i) {
        const int2 t = ctx->h_tile[i >> kTileShift];
        if ((long long)i < t.y) slot_of[(size_t)ctx->h_box[t.x].in0 + (size_t)tag[i]] = (long long)i;
    }
    std::vector<unsigned> words((size_t)v.W);
    std::vector<int> entries((size_t)v.cap_c);
    std::vector<int> crow((size_t)v.Mcap);
    for (int k = 0; k < m; ++k) {
        const size_t i = (size_t)slot_of[(size_t)which[k]];
        int cnt = 0;
        CK(cudaMemcpy(&cnt, (kind == 0 ? v.n_core : v.n_shell) + i, 4, cudaMemcpyDeviceToHost));
        if (cnt > cap) {
            set_err(ctx, "row %lld has %d entries, more than cap %d", which[k], cnt, cap);
            return RBL_EOVERFLOW;
        }
        counts[k] = cnt;
        int *out = rows + (size_t)k * cap;
        if (kind == 1 && v.full_list) { // row i of core[N][cap_c]
            const int n = cnt < v.cap_c ? cnt : v.cap_c;
            if (n > 0) CK(cudaMemcpy(entries.data(), v.core + i * (size_t)v.cap_c, 4 * (size_t)n, cudaMemcpyDeviceToHost));
            for (int q = 0; q < n; ++q) out[q] = tag[entries[q]];
            continue;
        }
        if (kind == 0) {
            // column i of core[cap_c][N]
            const int nc = cnt < v.cap_c ? cnt : v.cap_c;
            if (nc > 0)
                CK(cudaMemcpy2D(entries.data(), 4, v.core + i, 4 * N, 4, (size_t)nc, cudaMemcpyDeviceToHost));
            for (int q = 0; q < nc; ++q) out[q] = tag[entries[q]];
            continue;
        }
        if (v.W == 0) continue; // no masks (stencil pool)
        // bit b of mask word w is entry 32 w + b of the home cell's culled table
        int hc = 0;
        CK(cudaMemcpy(&hc, v.hcell + i, 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(crow.data(), v.ctab + (size_t)hc * v.Mcap, 4 * (size_t)v.Mcap, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy2D(words.data(), 4, v.mask + i, 4 * N, 4, (size_t)v.W, cudaMemcpyDeviceToHost));
        int q = 0;
        for (int w = 0; w < v.W && q < cnt; ++w) {
            unsigned word = words[w];
            while (word) {
                int bit = __builtin_ctz(word);
                word &= word - 1u;
                out[q++] = tag[crow[(w << 5) + bit]];
            }
        }
    }
    return RBL_OK;
}

rbl_status rbl_get_batch(rbl_ctx *ctx, long long step, int *batch, int *counts)
{
    if (!ctx || !batch || !counts || step < 0) return RBL_EINVAL;
    if (ctx->view.full_list) {
        set_err(ctx, "the full list draws no batches");
        return RBL_EINVAL;
    }
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    const View &v = ctx->view;
    const size_t N = (size_t)v.N;
    int *dj = (int *)v.staging;
    int *dn = dj + N * (size_t)v.p;
    CK(launch_batch(v, (unsigned long long)step, dj, dn, ctx->stream));
    st = check_flags(ctx);
    if (st != RBL_OK) return st;
    std::vector<int> tag(N), jj(N * (size_t)v.p), nb(N);
    CK(cudaMemcpy(tag.data(), v.tag, 4 * N, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(jj.data(), dj, 4 * N * (size_t)v.p, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nb.data(), dn, 4 * N, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < N; ++i) {
        const int2 tl = ctx->h_tile[i >> kTileShift];
        if ((long long)i >= tl.y) continue;
        const size_t t = (size_t)ctx->h_box[tl.x].in0 + (size_t)tag[i];
        counts[t] = nb[i];
        for (int q = 0; q < nb[i]; ++q) batch[t * v.p + q] = tag[jj[i * v.p + q]];
    }
    return RBL_OK;
}

rbl_status rbl_rdf(rbl_ctx *ctx, float dr, int nbins, long long *hist)
{
    if (!ctx || !hist || nbins < 1 || !(dr > 0.0f)) return RBL_EINVAL;
    if ((double)nbins * dr > ctx->prm.r_s) {
        set_err(ctx, "nbins * dr = %g exceeds r_s = %g", (double)nbins * dr, ctx->prm.r_s);
        return RBL_EINVAL;
    }
    const size_t nh = (size_t)nbins * (size_t)ctx->R;
    if (nh * 8 > ctx->staging_bytes) {
        set_err(ctx, "too many bins for the staging area");
        return RBL_EINVAL;
    }
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    unsigned long long *dh = (unsigned long long *)ctx->view.staging;
    CK(cudaMemsetAsync(dh, 0, 8 * nh, ctx->stream));
    CK(launch_rdf(ctx->view, dr, nbins, dh, ctx->stream));
    std::vector<unsigned long long> h(nh);
    CK(cudaMemcpyAsync(h.data(), dh, 8 * nh, cudaMemcpyDeviceToHost, ctx->stream));
    st = check_flags(ctx);
    if (st != RBL_OK) return st;
    for (size_t b = 0; b < nh; ++b) hist[b] += (long long)h[b];
    return RBL_OK;
}

rbl_status rbl_density_profile(rbl_ctx *ctx, int axis, int nbins, long long *hist)
{
    if (!ctx || !hist || axis < 0 || axis > 2 || nbins < 1 || nbins > kMaxProfileBins) return RBL_EINVAL;
    const size_t nh = (size_t)nbins * (size_t)ctx->R;
    if (nh * 8 > ctx->staging_bytes) {
        set_err(ctx, "too many bins for the staging area");
        return RBL_EINVAL;
    }
    unsigned long long *dh = (unsigned long long *)ctx->view.staging;
    CK(cudaMemsetAsync(dh, 0, 8 * nh, ctx->stream));
    CK(launch_profile(ctx->view, axis, nbins, dh, ctx->stream));
    std::vector<unsigned long long> h(nh);
    CK(cudaMemcpyAsync(h.data(), dh, 8 * nh, cudaMemcpyDeviceToHost, ctx->stream));
    rbl_status st = check_flags(ctx);
    if (st != RBL_OK) return st;
    for (size_t b = 0; b < nh; ++b) hist[b] += (long long)h[b];
    return RBL_OK;
}

rbl_status rbl_set_launch_config(rbl_ctx *ctx, int force_threads, int build_warps)
{
    if (!ctx) return RBL_EINVAL;
    if (force_threads != 64 && force_threads != 128 && force_threads != 256) {
        set_err(ctx, "force_threads must be 64, 128 or 256 (got %d)", force_threads);
        return RBL_EINVAL;
    }
    if (build_warps != 2 && build_warps != 4 && build_warps != 8) {
        set_err(ctx, "build_warps must be 2, 4 or 8 (got %d)", build_warps);
        return RBL_EINVAL;
    }
    if (ctx->view.force_threads != force_threads || ctx->view.build_warps != build_warps) {
        ctx->view.force_threads = force_threads;
        ctx->view.build_warps = build_warps;
        drop_graphs(ctx); // the captured steps hold the old launch shapes
    }
    return RBL_OK;
}

rbl_status rbl_autotune(rbl_ctx *ctx, int trials, int *force_threads, int *build_warps)
{
    if (!ctx || trials < 1) return RBL_EINVAL;
    rbl_status st = ensure_lists(ctx);
    if (st != RBL_OK) return st;
    // the trials rebuild and re-evaluate: keep the per-replica scalars (rebuild
    // counts, build statistics, energies) as they were
    st = read_scalars(ctx, true);
    if (st != RBL_OK) return st;
    std::vector<RepScalars> saved(ctx->h_rs, ctx->h_rs + ctx->R);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int ft[3] = {64, 128, 256}, bw[3] = {2, 4, 8};
    float best_f = 1e30f, best_b = 1e30f;
    int pick_f = ctx->view.force_threads, pick_b = ctx->view.build_warps;
    cudaError_t e = cudaSuccess;
    // List build, timed on the images of the last build (ubuild) in place of the
    // current ones: the particles are already in that build's cell order, so the
    // permutation is the identity and the lists come out as they were; the current
    // images and the trajectory are untouched.
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        View v = ctx->view;
        v.build_warps = bw[k];
        v.pos = v.ubuild;
        e = launch_rebuild(v, ctx->n_scan_blocks, false, ctx->stream); // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        for (int t = 0; t < trials && e == cudaSuccess; ++t)
            e = launch_rebuild(v, ctx->n_scan_blocks, false, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_b) {
            best_b = ms;
            pick_b = bw[k];
        }
    }
    // force kernel and its reduction (the step counter is not advanced)
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        View v = ctx->view;
        v.force_threads = ft[k];
        e = launch_forces(v, 0, 0, false, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        for (int t = 0; t < trials && e == cudaSuccess; ++t) e = launch_forces(v, 0, 0, false, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_f) {
            best_f = ms;
            pick_f = ft[k];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_err(ctx, "autotune failed: %s", cudaGetErrorString(e));
        return RBL_ECUDA;
    }
    CK(cudaMemcpyAsync(ctx->view.rs, saved.data(), sizeof(RepScalars) * (size_t)ctx->R, cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->force_valid = 0;
    ctx->energy_valid = 0;
    st = rbl_set_launch_config(ctx, pick_f, pick_b);
    if (st != RBL_OK) return st;
    if (force_threads) *force_threads = pick_f;
    if (build_warps) *build_warps = pick_b;
    return check_flags(ctx);
}

// Cell size by measurement.  K sets the cell stencil, hence the canonical row order and
// which batch each step draws, so it is chosen before a run from timings of the
// caller's own system, each K in a context of its own (launch shapes tuned for it).
rbl_status rbl_tune_cells_workspace_size(const rbl_params *prm, int N, size_t *bytes)
{
    if (!prm || !bytes) return RBL_EINVAL;
    size_t best = 0;
    for (int K = 1; K <= 3; ++K) {
        rbl_params q = *prm;
        q.cells_per_cutoff = K;
        size_t b = 0;
        if (rbl_workspace_size(&q, N, &b) == RBL_OK && b > best) best = b;
    }
    if (best == 0) return RBL_EINVAL;
    *bytes = best;
    return RBL_OK;
}

rbl_status rbl_tune_cells(const rbl_params *prm, int N, const double *x, const double *v, void *workspace,
                          size_t workspace_bytes, void *stream, int steps, int *K_best, float *ms_per_step)
{
    if (!prm || !x || !workspace || !K_best || steps < 1) return RBL_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return RBL_ECUDA;
    }
    rbl_status st = RBL_OK;
    float best = 0.f;
    int pick = 0;
    for (int K = 1; K <= 3 && st == RBL_OK; ++K) {
        float ms = -1.f; // not valid for these parameters, or larger than the workspace
        rbl_params q = *prm;
        q.cells_per_cutoff = K;
        size_t need = 0;
        if (rbl_workspace_size(&q, N, &need) == RBL_OK && need <= workspace_bytes) {
            rbl_ctx *ctx = nullptr;
            st = rbl_create(&q, N, workspace, workspace_bytes, stream, &ctx);
            if (st == RBL_OK) st = rbl_set_state(ctx, x, v, 0, 0);
            if (st == RBL_OK) st = rbl_autotune(ctx, 2, nullptr, nullptr);
            if (st == RBL_OK) st = rbl_step(ctx, steps); // warm-up, rebuilds included
            if (st == RBL_OK) {
                if (cudaEventRecord(e0, s) != cudaSuccess) st = RBL_ECUDA;
                if (st == RBL_OK) st = rbl_step_async(ctx, steps);
                if (st == RBL_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                    st = RBL_ECUDA;
                float t = 0.f;
                if (st == RBL_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = RBL_ECUDA;
                rbl_obs o;
                if (st == RBL_OK) st = rbl_observables(ctx, &o); // waits; reports the timed steps' device flags
                ms = t / (float)steps;
            }
            if (ctx) rbl_destroy(ctx);
            if (st == RBL_OK && (pick == 0 || ms < best)) {
                best = ms;
                pick = K;
            }
        }
        if (ms_per_step) ms_per_step[K - 1] = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    if (st != RBL_OK) return st;
    if (pick == 0) return RBL_EINVAL;
    *K_best = pick;
    return RBL_OK;
}

rbl_status rbl_set_phase_timing(rbl_ctx *ctx, int enable)
{
    if (!ctx) return RBL_EINVAL;
    ctx->phase_timing = enable ? 1 : 0;
    return RBL_OK;
}

rbl_status rbl_phase_times(rbl_ctx *ctx, double ms[5], long long *steps, int reset)
{
    if (!ctx) return RBL_EINVAL;
    if (ms)
        for (int k = 0; k < kPhases; ++k) ms[k] = ctx->phase_ms[k];
    if (steps) *steps = ctx->phase_steps;
    if (reset) {
        for (int k = 0; k < kPhases; ++k) ctx->phase_ms[k] = 0.0;
        ctx->phase_steps = 0;
    }
    return RBL_OK;
}

rbl_status rbl_rebuild_times(rbl_ctx *ctx, double ms[2], long long *rebuilds, int reset)
{
    if (!ctx) return RBL_EINVAL;
    if (ms)
        for (int k = 0; k < 2; ++k) ms[k] = ctx->rebuild_ms[k];
    if (rebuilds) *rebuilds = ctx->rebuild_n;
    if (reset) {
        ctx->rebuild_ms[0] = ctx->rebuild_ms[1] = 0.0;
        ctx->rebuild_n = 0;
    }
    return RBL_OK;
}

void rbl_destroy(rbl_ctx *ctx)
{
    if (!ctx) return;
    drop_graphs(ctx);
    for (int k = 0; k < ctx->ev_cap * kPhaseEvents; ++k) cudaEventDestroy(ctx->ev[k]);
    std::free(ctx->ev);
    for (int k = 0; k < 3; ++k)
        if (ctx->rb_ev[k]) cudaEventDestroy(ctx->rb_ev[k]);
    delete ctx->h_sc;
    delete[] ctx->h_rs;
    delete[] ctx->h_box;
    delete[] ctx->h_tile;
    delete[] ctx->h_cell_rep;
    delete ctx;
}

const char *rbl_last_error(const rbl_ctx *ctx) { return ctx ? ctx->err : "null context"; }

const char *rbl_status_string(rbl_status s)
{
    switch (s) {
    case RBL_OK: return "RBL_OK";
    case RBL_EINVAL: return "RBL_EINVAL";
    case RBL_ENOMEM: return "RBL_ENOMEM";
    case RBL_EOVERFLOW: return "RBL_EOVERFLOW";
    case RBL_ENONFINITE: return "RBL_ENONFINITE";
    case RBL_ETIMEOUT: return "RBL_ETIMEOUT";
    case RBL_ECUDA: return "RBL_ECUDA";
    }
    return "unknown";
}

} // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free force evaluation.
//
// Some callers cannot allocate device memory at the point where they need forces:
// a plugin called from inside another engine's time step, where the host
// application owns all device memory through its own pool and forbids cudaMalloc
// (which can fail or synchronise the device mid-run), or code that runs after its
// initialisation phase under a no-allocation rule.  rbl_forces_static serves them:
// every array it needs lives in one file-scope device array of fixed size, loaded
// with the library, so the call allocates nothing, host or device.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = (size_t)48 << 20; // 48 MiB, held by every device that loads the library
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_ptr[kMaxDevices]; // device address of g_static_scratch, per device ordinal

// Device address of the scratch array on the current device.  The host-side name
// g_static_scratch is only a stand-in; the address comes from cudaGetSymbolAddress
// with that device current.  The first call on a device sets it up (loading the
// module there); it is looked up again on every call, so a device reset that reloads
// the module (and may move the array) leaves no stale address behind.
rbl_status static_scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return RBL_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return RBL_EINVAL;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return RBL_ECUDA;
    }
    g_static_ptr[dev] = p;
    *out = p;
    return RBL_OK;
}
} // namespace

extern "C" rbl_status rbl_forces_static(const rbl_params *prm, int N, const double *x, long long step, double *F,
                                        void *stream)
{
    if (!x || !F || step < 0) return RBL_EINVAL;
    rbl_status st = validate_batch(prm, 1, &N, nullptr, 0);
    if (st != RBL_OK) return st;
    if (prm->potential != RBL_POT_LJ) return RBL_EINVAL; // no charges can be passed here
    const Plan P = make_plan(prm, 1, &N);
    if (P.total > kStaticScratchBytes) return RBL_ENOMEM;
    void *base = nullptr;
    st = static_scratch_address(&base);
    if (st != RBL_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    View v;
    assign_view(v, prm, P, (char *)base);
    const Box b = make_box(prm, N, 0, 0, 0);
    // the array keeps the previous call's contents: rewrite the tables and reset the
    // scalars this call reads
    DevScalars h{};
    h.step = (unsigned long long)step;
    if (launch_init_single(v, b, s) != cudaSuccess) return RBL_ECUDA;
    if (cudaMemcpyAsync(v.sc, &h, sizeof(DevScalars), cudaMemcpyHostToDevice, s) != cudaSuccess) return RBL_ECUDA;
    if (cudaMemsetAsync(v.rs, 0, sizeof(RepScalars), s) != cudaSuccess) return RBL_ECUDA;
    if (launch_load_state(v, x, nullptr, s) != cudaSuccess) return RBL_ECUDA;
    if (launch_rebuild(v, P.n_scan_blocks, false, s) != cudaSuccess) return RBL_ECUDA;
    if (launch_forces(v, 0, 0, false, s) != cudaSuccess) return RBL_ECUDA;
    if (launch_store_forces(v, F, s) != cudaSuccess) return RBL_ECUDA;
    if (cudaMemcpyAsync(&h, v.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RBL_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RBL_ECUDA;
    if (h.flags & (kFlagOverflow | kFlagCellOverflow)) return RBL_EOVERFLOW;
    if (h.flags & kFlagNonFinite) return RBL_ENONFINITE;
    if (h.flags & kFlagRngLimit) return RBL_ETIMEOUT;
    return RBL_OK;
}
