// lbm_api.cu -- host side of the C ABI declared in include/lbm.h: context
// creation (cell flags, edge-cell list, device memory layout), the time loop
// with its epilogue schedule (time average, snapshots, obstacle force), read
// and write of the state, checkpoints.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

constexpr size_t ALIGN = 256;
size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

size_t storage_bytes(int s) { return s == LBM_F64 ? 8 : (s == LBM_F32 ? 4 : 2); }

// Device memory layout of a context (byte offsets into one allocation).
struct Layout {
    int64_t n = 0, slot = 0, n_half = 0, snap_cells = 0;
    size_t pdf = 0, flags = 0, edge = 0, ub = 0, ob = 0, msum = 0, snaps = 0, stage = 0, force = 0,
           fpart = 0, fcount = 0, tpart = 0, tout = 0, status = 0, total = 0;
    int tot_blocks = 0;
};

// Bytes of the time-average sums: [4][n] doubles, plus [6][n] velocity
// products with turbulence statistics on.
size_t msum_bytes(const lbm_params &p, int64_t n)
{
    return p.mean_every > 0 ? (size_t)(p.stats ? 10 : 4) * n * 8 : 0;
}

// Upper bound of the edge-cell count: every cell on a domain face, plus the
// (at most 26) fluid neighbours of each solid cell.
int64_t edge_bound(const lbm_grid &g, int64_t n_solid)
{
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    int64_t inner = 1;
    for (int d : {g.nx, g.ny, g.nz}) inner *= (d > 2 ? d - 2 : 0);
    return std::min<int64_t>(n, (n - inner) + 26 * n_solid) + 1;
}

Layout make_layout(const lbm_grid &g, const lbm_params &p, int64_t n_solid)
{
    Layout L;
    L.n = (int64_t)g.nx * g.ny * g.nz;
    L.slot = (L.n + 63) / 64 * 64;
    L.n_half = (int64_t)((g.nx + 1) / 2) * ((g.ny + 1) / 2) * ((g.nz + 1) / 2);
    L.snap_cells = p.snap_halfres ? L.n_half : L.n;
    const size_t rsz = p.storage == LBM_F64 ? 8 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L.pdf = take((size_t)Q * L.slot * storage_bytes(p.storage));
    L.flags = take((size_t)L.n);
    L.edge = take((size_t)edge_bound(g, n_solid) * 16);
    L.ub = take((size_t)3 * g.ny * g.nz * rsz);
    L.ob = take(p.face_x_hi == LBM_FACE_OUTFLOW ? (size_t)18 * g.ny * g.nz * rsz : 0);
    L.msum = take(msum_bytes(p, L.n));
    L.snaps = take(p.snap_count > 0 ? (size_t)p.snap_count * 4 * L.snap_cells * 4 : 0);
    L.stage = take(p.snap_count > 0 && p.snap_halfres ? (size_t)4 * L.n * 4 : 0);
    const int64_t cap = p.force_capacity > 0 ? p.force_capacity : 65536;
    L.force = take(p.force_every > 0 ? (size_t)cap * 3 * 8 : 0);
    L.fpart = take((size_t)3 * 8 * ((L.n + EDGE_BLOCK - 1) / EDGE_BLOCK + 1));
    L.fcount = take(sizeof(unsigned));
    L.tot_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((L.n + 255) / 256, gb300::sm_count() * 8));
    L.tpart = take((size_t)4 * 8 * L.tot_blocks);
    L.tout = take(4 * 8);
    L.status = take(sizeof(int));
    L.total = off;
    return L;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace lbm {
// Message for lbm_last_error(NULL) from entry points defined in other units.
void set_global_error(const std::string &m) { g_err = m; }
}  // namespace lbm

// Fourth-order parametrisation (Sec. 3.2; Geier, Pasquali & Schoenherr 2017):
// the published rates omega3 (sums of third-order pairs), omega4 (their
// differences), omega5 (C_111) and the factors of the fourth-order equilibria,
// as functions of the shear rate w1 and the bulk rate w2; out = {omega3,
// omega4, omega5, -(2/3) A (1/w1 - 1/2), B (1 - w1/2), lambda}.
static void param4_factors(double w1, double w2, double lambda, double out[6])
{
    const double w1s = w1 * w1, w2s = w2 * w2;
    out[0] = 8.0 * (w1 - 2.0) * (w2 * (3.0 * w1 - 1.0) - 5.0 * w1) /
             (8.0 * (5.0 - 2.0 * w1) * w1 + w2 * (8.0 + w1 * (9.0 * w1 - 26.0)));
    out[1] = 8.0 * (w1 - 2.0) * (w1 + w2 * (3.0 * w1 - 7.0)) / (w2 * (56.0 - 42.0 * w1 + 9.0 * w1s) - 8.0 * w1);
    out[2] = 24.0 * (w1 - 2.0) * (4.0 * w1s + w1 * w2 * (18.0 - 13.0 * w1) + w2s * (2.0 + w1 * (6.0 * w1 - 11.0))) /
             (16.0 * w1s * (w1 - 6.0) - 2.0 * w1 * w2 * (216.0 + 5.0 * w1 * (9.0 * w1 - 46.0)) +
              w2s * (w1 * (3.0 * w1 - 10.0) * (15.0 * w1 - 28.0) - 48.0));
    const double den = (w1 - w2) * (w2 * (2.0 + 3.0 * w1) - 8.0 * w1);
    const double A = (4.0 * w1s + 2.0 * w1 * w2 * (w1 - 6.0) + w2s * (w1 * (10.0 - 3.0 * w1) - 4.0)) / den;
    const double B = (4.0 * w1 * w2 * (9.0 * w1 - 16.0) - 4.0 * w1s - 2.0 * w2s * (2.0 + 9.0 * w1 * (w1 - 2.0))) / (3.0 * den);
    out[3] = -(2.0 / 3.0) * A * (1.0 / w1 - 0.5);
    out[4] = B * (1.0 - 0.5 * w1);
    out[5] = lambda;
}

struct lbm_ctx {
    lbm_grid g;
    lbm_params p;
    Layout L;
    cudaStream_t stream = nullptr;
    bool owns = false;
    char *base = nullptr;
    int64_t n_edge = 0;
    int64_t t = 0;
    double w1 = 0;
    bool plain = true;
    int block_x = 128, block_y = 1;
    int64_t msamples = 0;
    std::vector<char> snap_taken;
    std::vector<double> force_host;   // flushed rows (deviation part)
    int64_t force_rows_dev = 0, force_cap = 0;
    double force_w[3] = {0, 0, 0};    // constant w-part of the obstacle force
    bool unstable = false;
    bool in_batch = false;
    // interpolated bounce-back links (device, owned by the context)
    uint4 *qlinks = nullptr;
    double *qval = nullptr, *qpart = nullptr;
    unsigned *qcount = nullptr;
    int64_t n_qlinks = 0;
    // probes: (u, v, w, p) at listed cells every probe_every steps
    int64_t *probe_cells = nullptr;
    float *probe_ring = nullptr;
    int64_t n_probes = 0, probe_every = 1, probe_cap = 0, probe_rows_dev = 0;
    std::vector<float> probe_host;
    // monitor plane (Sec. 2): (u, v, w, p) of the plane z = plane_z every
    // plane_every steps, a device ring of plane_cap planes flushed to the host
    int plane_z = -1;
    float *plane_ring = nullptr;
    int64_t plane_every = 1, plane_cap = 0, plane_rows_dev = 0;
    std::vector<float> plane_host;
    std::vector<int64_t> plane_steps;
    std::string err;
    int64_t n_fluid = 0, n_bulk = 0, n_wall = 0, launches = 0;
    // kernel timing: events recorded per step (start, mid, end) and the step kind
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_kind;

    template <class T> T *at(size_t off) { return reinterpret_cast<T *>(base + off); }

    StepArgs args()
    {
        StepArgs a{};
        a.pdf = base + L.pdf;
        a.slot = L.slot;
        a.flags = at<uint8_t>(L.flags);
        a.edge = at<uint4>(L.edge);
        a.n_edge = n_edge;
        a.n_wall = n_wall;
        a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
        a.nxy = (int64_t)g.nx * g.ny;
        a.n = L.n;
        a.w1 = w1; a.w2 = p.omega_bulk; a.w3 = p.omega_higher;
        a.galilean = p.galilean_correction;
        a.face_x_lo = p.face_x_lo; a.face_x_hi = p.face_x_hi; a.face_y = p.face_y; a.face_z = p.face_z;
        a.u_in = p.u_in; a.rho_in = p.rho_in; a.rho_out = p.rho_out;
        a.w1f = (float)a.w1; a.w2f = (float)a.w2; a.w3f = (float)a.w3;
        a.param4 = p.param4 ? 1 : 0;
        a.xface_bulk = p.xface_edge ? 0 : 1;
        if (a.param4) param4_factors(a.w1, a.w2, p.limiter, a.p4);
        for (int k = 0; k < 6; ++k) a.p4f[k] = (float)a.p4[k];
        const int64_t es = (int64_t)storage_bytes(p.storage);
        for (int i = 0; i < Q; ++i) {
            const int64_t off = cx_of(i) + (int64_t)cy_of(i) * g.nx + (int64_t)cz_of(i) * a.nxy;
            a.boff[0][i] = (int64_t)i * L.slot * es;                   // even: own slot i
            a.boff[1][i] = (int64_t)(Q - 1 - i) * L.slot * es;         // even: own slot 26-i
            a.boff[2][i] = ((int64_t)(Q - 1 - i) * L.slot - off) * es; // odd: slot 26-i of x - c_i
            a.boff[3][i] = ((int64_t)i * L.slot + off) * es;           // odd: slot i of x + c_i
        }
        a.u_in_f = (float)a.u_in; a.rho_in_f = (float)a.rho_in; a.rho_out_f = (float)a.rho_out;
        a.ub = base + L.ub;
        a.stats = p.stats ? 1 : 0;
        a.qlinks = qlinks;
        a.qval = qval;
        a.n_qlinks = n_qlinks;
        a.qpart = qpart;
        a.qcount = qcount;
        a.ob = base + L.ob;
        a.fcount = at<unsigned>(L.fcount);
        a.status = at<int>(L.status);
        return a;
    }
};

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
            return LBM_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

static lbm_status fail(lbm_ctx *ctx, lbm_status s, const std::string &m)
{
    if (ctx) ctx->err = m; else g_err = m;
    return s;
}

// ---------------------------------------------------------------------------
extern "C" void lbm_params_default(lbm_params *p)
{
    std::memset(p, 0, sizeof(*p));
    p->re = 1000.0; p->u_in = 0.05; p->l_ref = 1.0;
    p->omega1 = 0.0; p->omega_bulk = 1.0; p->omega_higher = 1.0;
    p->rho_in = 1.0; p->rho_out = 1.0;
    p->storage = LBM_F32; p->galilean_correction = 1;
    p->face_x_lo = LBM_FACE_INLET; p->face_x_hi = LBM_FACE_OUTFLOW;
    p->face_y = LBM_FACE_WALL; p->face_z = LBM_FACE_WALL;
    p->force_capacity = 65536;
    p->param4 = 0; p->limiter = 0.01;
}

static std::string validate(const lbm_grid *g, const lbm_params *p)
{
    if (!g || !p) return "null grid or params";
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return "grid dimensions must be >= 1";
    if (g->ny > 65535 || g->nz > 65535) return "ny and nz must be <= 65535";
    if ((int64_t)g->nx * g->ny * g->nz >= (int64_t(1) << 32)) return "grid must have fewer than 2^32 cells";
    if (p->storage < LBM_F64 || p->storage > LBM_F16C) return "unknown storage";
    if (p->face_x_lo != LBM_FACE_INLET && p->face_x_lo != LBM_FACE_WALL && p->face_x_lo != LBM_FACE_PERIODIC)
        return "face_x_lo must be inlet, wall or periodic";
    if (p->face_x_hi != LBM_FACE_OUTLET && p->face_x_hi != LBM_FACE_OUTFLOW && p->face_x_hi != LBM_FACE_WALL &&
        p->face_x_hi != LBM_FACE_PERIODIC)
        return "face_x_hi must be outflow, outlet, wall or periodic";
    if ((p->face_x_lo == LBM_FACE_PERIODIC) != (p->face_x_hi == LBM_FACE_PERIODIC))
        return "periodic x needs both x faces periodic";
    if ((p->face_y != LBM_FACE_WALL && p->face_y != LBM_FACE_PERIODIC) ||
        (p->face_z != LBM_FACE_WALL && p->face_z != LBM_FACE_PERIODIC))
        return "y and z faces must be wall or periodic";
    if (p->omega1 <= 0 && !(p->re > 0 && p->u_in >= 0 && p->l_ref > 0)) return "need omega1 > 0 or re, l_ref > 0";
    if (p->mean_every < 0 || p->snap_count < 0 || p->force_every < 0) return "negative schedule";
    if (p->snap_count > 0 && p->snap_every < 1) return "snap_every must be >= 1";
    if (p->block_x != 0 && (p->block_x % 32 != 0 || p->block_x > 256)) return "block_x must be a multiple of 32, <= 256";
    if (p->block_y < 0 || (p->block_x ? p->block_x : 128) * (p->block_y ? p->block_y : 1) > 256)
        return "block_x * block_y must be <= 256";
    if (p->param4 != 0 && p->param4 != 1) return "param4 must be 0 or 1";
    if (p->xface_edge != 0 && p->xface_edge != 1) return "xface_edge must be 0 or 1";
    if (p->param4) {
        if (!(p->limiter > 0.0)) return "param4 needs limiter > 0";
        const double w1 = p->omega1 > 0 ? p->omega1 : 1.0 / (3.0 * p->u_in * p->l_ref / p->re + 0.5);
        if (std::fabs(w1 - p->omega_bulk) < 1e-9)
            return "param4 is undefined at omega1 = omega_bulk (choose another bulk rate)";
    }
    return "";
}

// Number of solid cells of a host or device mask (0 for NULL); -1 on error.
static int64_t count_solid(const uint8_t *mask, int64_t n)
{
    if (!mask) return 0;
    std::vector<uint8_t> h;
    const uint8_t *m = mask;
    if (is_device_ptr(mask)) {
        h.resize(n);
        if (cudaMemcpy(h.data(), mask, n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        m = h.data();
    }
    int64_t k = 0;
    for (int64_t c = 0; c < n; ++c) k += (m[c] != 0);
    return k;
}

extern "C" size_t lbm_workspace_bytes(const lbm_grid *g, const uint8_t *mask, const lbm_params *p)
{
    if (!validate(g, p).empty()) return 0;
    const int64_t ns = count_solid(mask, (int64_t)g->nx * g->ny * g->nz);
    if (ns < 0) return 0;
    return make_layout(*g, *p, ns).total;
}

static lbm_status create_impl(const lbm_grid *g, const uint8_t *mask, const lbm_params *p, void *stream,
                              void *workspace, size_t ws_bytes, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is null");
    *out = nullptr;
    std::string v = validate(g, p);
    if (!v.empty()) return fail(nullptr, LBM_ERR_ARG, v);
    lbm_ctx *ctx = new lbm_ctx();
    ctx->g = *g;
    ctx->p = *p;
    if (ctx->p.force_capacity <= 0) ctx->p.force_capacity = 65536;
    const int64_t n_solid = count_solid(mask, (int64_t)g->nx * g->ny * g->nz);
    if (n_solid < 0) {
        delete ctx;
        return fail(nullptr, LBM_ERR_CUDA, "mask could not be read");
    }
    ctx->L = make_layout(*g, ctx->p, n_solid);
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->w1 = p->omega1 > 0 ? p->omega1 : 1.0 / (3.0 * p->u_in * p->l_ref / p->re + 0.5);
    ctx->plain = (p->omega_higher == 1.0) && !p->param4;
    ctx->block_x = p->block_x ? p->block_x : 128;
    ctx->block_y = p->block_y ? p->block_y : 1;
    ctx->force_cap = ctx->p.force_capacity;
    ctx->snap_taken.assign(std::max<int64_t>(0, p->snap_count), 0);
    const Layout &L = ctx->L;
    auto bail = [&](lbm_status s) {
        g_err = ctx->err;
        if (ctx->owns && ctx->base) cudaFree(ctx->base);
        delete ctx;
        return s;
    };
    if (workspace) {
        if (ws_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % ALIGN) != 0) {
            ctx->err = "workspace too small or not 256-byte aligned";
            return bail(LBM_ERR_OOM);
        }
        ctx->base = static_cast<char *>(workspace);
    } else {
        cudaError_t e = cudaMalloc(&ctx->base, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->err = std::string("cudaMalloc of ") + std::to_string(L.total) + " bytes failed";
            return bail(LBM_ERR_OOM);
        }
        ctx->owns = true;
    }
    cudaStream_t s = ctx->stream;
    const int64_t n = L.n;
    // the mask goes through the (not yet used) population region
    uint8_t *dmask = nullptr;
    if (mask) {
        dmask = ctx->at<uint8_t>(L.pdf);
        if (cudaMemcpyAsync(dmask, mask, n, is_device_ptr(mask) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess) {
            ctx->err = "mask upload failed";
            return bail(LBM_ERR_CUDA);
        }
    }
    launch_flags(dmask, ctx->at<uint8_t>(L.flags), g->nx, g->ny, g->nz,
                 p->face_x_lo != LBM_FACE_PERIODIC && !p->xface_edge, p->face_x_hi != LBM_FACE_PERIODIC && !p->xface_edge,
                 p->face_y == LBM_FACE_WALL, p->face_z == LBM_FACE_WALL, s);
    // boundary-cell records on the device (ascending cell order keeps rows
    // contiguous): cell index and the link code of each of the 27 directions
    // in the pull view (where population i of the cell comes from); the
    // scratch (chunk counts and offsets, solid links per direction) sits in
    // the population array behind the uploaded mask, before it is cleared
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const int64_t nb = record_blocks(n);
    unsigned char *scr = reinterpret_cast<unsigned char *>(ctx->base + L.pdf) + ((n + 255) / 256) * 256;
    int *dcounts = reinterpret_cast<int *>(scr);
    int64_t *doffs = reinterpret_cast<int64_t *>(scr + ((nb * 16 + 255) / 256) * 256);
    unsigned long long *dsolid = reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(doffs) +
                                                                         ((nb * 8 + 255) / 256) * 256);
    std::vector<int> hcounts((size_t)nb * 4);
    launch_record_count(ctx->at<uint8_t>(L.flags), n, dcounts, s);
    if (cudaMemcpyAsync(hcounts.data(), dcounts, hcounts.size() * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        ctx->err = std::string("flag build failed: ") + cudaGetErrorString(cudaGetLastError());
        return bail(LBM_ERR_CUDA);
    }
    std::vector<int64_t> hoffs((size_t)nb);
    int64_t n_edge = 0;
    for (int64_t b = 0; b < nb; ++b) {
        ctx->n_fluid += hcounts[4 * b];
        ctx->n_bulk += hcounts[4 * b + 1];
        ctx->n_wall += hcounts[4 * b + 2];
        hoffs[b] = n_edge;
        n_edge += hcounts[4 * b + 3];
    }
    if (n_edge > edge_bound(*g, n_solid)) {
        ctx->err = "edge-cell count exceeds its bound";
        return bail(LBM_ERR_OOM);
    }
    ctx->n_edge = n_edge;
    unsigned long long hsolid[Q] = {};
    if (cudaMemcpyAsync(doffs, hoffs.data(), hoffs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(dsolid, 0, sizeof(hsolid), s) != cudaSuccess) {
        ctx->err = "edge list build failed";
        return bail(LBM_ERR_CUDA);
    }
    launch_record_write(ctx->at<uint8_t>(L.flags), nx, ny, nz, p->face_x_lo, p->face_x_hi, p->face_y, p->face_z, doffs,
                        ctx->at<uint4>(L.edge), dsolid, s);
    if (cudaMemcpyAsync(hsolid, dsolid, sizeof(hsolid), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        ctx->err = std::string("edge list build failed: ") + cudaGetErrorString(cudaGetLastError());
        return bail(LBM_ERR_CUDA);
    }
    // the constant part sum 2 c_j w_j of the obstacle force over the links
    // heading into the obstacle, from the exact per-direction counts
    for (int j = 0; j < Q; ++j) {
        ctx->force_w[0] += 2.0 * cx_of(j) * w_of(j) * (double)hsolid[j];
        ctx->force_w[1] += 2.0 * cy_of(j) * w_of(j) * (double)hsolid[j];
        ctx->force_w[2] += 2.0 * cz_of(j) * w_of(j) * (double)hsolid[j];
    }
    // state at rest (shifted populations 0), accumulators cleared
    bool ok = cudaMemsetAsync(ctx->base + L.pdf, 0, (size_t)Q * L.slot * storage_bytes(p->storage), s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(ctx->base + L.ub, 0, (size_t)3 * ny * nz * (p->storage == LBM_F64 ? 8 : 4), s) == cudaSuccess;
    if (p->mean_every > 0) ok = ok && cudaMemsetAsync(ctx->base + L.msum, 0, msum_bytes(*p, n), s) == cudaSuccess;
    if (p->snap_count > 0) {
        ok = ok && cudaMemsetAsync(ctx->base + L.snaps, 0, (size_t)p->snap_count * 4 * L.snap_cells * 4, s) == cudaSuccess;
        if (p->snap_halfres) ok = ok && cudaMemsetAsync(ctx->base + L.stage, 0, (size_t)4 * n * 4, s) == cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(ctx->base + L.fcount, 0, sizeof(unsigned), s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(ctx->base + L.status, 0, sizeof(int), s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        ctx->err = std::string("initialisation failed: ") + cudaGetErrorString(cudaGetLastError());
        return bail(LBM_ERR_CUDA);
    }
    *out = ctx;
    return LBM_OK;
}

extern "C" lbm_status lbm_create(const lbm_grid *g, const uint8_t *mask, const lbm_params *p, void *stream,
                                 lbm_ctx **out)
{
    return create_impl(g, mask, p, stream, nullptr, 0, out);
}

extern "C" lbm_status lbm_create_in(const lbm_grid *g, const uint8_t *mask, const lbm_params *p, void *stream,
                                    void *workspace, size_t ws_bytes, lbm_ctx **out)
{
    if (!workspace) return fail(nullptr, LBM_ERR_ARG, "workspace is null");
    return create_impl(g, mask, p, stream, workspace, ws_bytes, out);
}

extern "C" lbm_status lbm_destroy(lbm_ctx *ctx)
{
    if (!ctx) return LBM_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    cudaFree(ctx->probe_cells);
    cudaFree(ctx->probe_ring);
    cudaFree(ctx->plane_ring);
    cudaFree(ctx->qlinks);
    cudaFree(ctx->qval);
    cudaFree(ctx->qpart);
    cudaFree(ctx->qcount);
    if (ctx->owns && ctx->base) cudaFree(ctx->base);
    delete ctx;
    return LBM_OK;
}

extern "C" int64_t lbm_time(const lbm_ctx *ctx) { return ctx ? ctx->t : -1; }

static lbm_status flush_forces(lbm_ctx *ctx)
{
    if (ctx->force_rows_dev == 0) return LBM_OK;
    const size_t old = ctx->force_host.size();
    ctx->force_host.resize(old + 3 * ctx->force_rows_dev);
    CK(cudaMemcpyAsync(ctx->force_host.data() + old, ctx->base + ctx->L.force,
                       sizeof(double) * 3 * ctx->force_rows_dev, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->force_rows_dev = 0;
    return LBM_OK;
}

static lbm_status flush_planes(lbm_ctx *ctx)
{
    if (ctx->plane_rows_dev == 0) return LBM_OK;
    const size_t per = (size_t)4 * ctx->g.nx * ctx->g.ny;
    const size_t old = ctx->plane_host.size(), cnt = per * ctx->plane_rows_dev;
    ctx->plane_host.resize(old + cnt);
    CK(cudaMemcpyAsync(ctx->plane_host.data() + old, ctx->plane_ring, sizeof(float) * cnt, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->plane_rows_dev = 0;
    return LBM_OK;
}

static lbm_status flush_probes(lbm_ctx *ctx)
{
    if (ctx->probe_rows_dev == 0) return LBM_OK;
    const size_t old = ctx->probe_host.size(), cnt = (size_t)4 * ctx->n_probes * ctx->probe_rows_dev;
    ctx->probe_host.resize(old + cnt);
    CK(cudaMemcpyAsync(ctx->probe_host.data() + old, ctx->probe_ring, sizeof(float) * cnt, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->probe_rows_dev = 0;
    return LBM_OK;
}

static cudaEvent_t next_event(lbm_ctx *ctx)
{
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_used++];
}

static void step_launch(lbm_ctx *ctx, const StepArgs &a, bool odd, bool epi)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
    if (ctx->timing) {
        e0 = next_event(ctx);
        e1 = next_event(ctx);
        e2 = next_event(ctx);
        e3 = next_event(ctx);
        if (e0 && e1 && e2 && e3) {
            cudaEventRecord(e0, ctx->stream);
            ctx->ev_kind.push_back((odd ? 1 : 0) + (epi ? 2 : 0));
        } else {
            e1 = e2 = nullptr;
        }
    }
    switch (ctx->p.storage) {
    case LBM_F64: launch_step_f64(a, odd, epi, ctx->plain, ctx->block_x, ctx->block_y, ctx->stream, e1, e2); break;
    case LBM_F32: launch_step_f32(a, odd, epi, ctx->plain, ctx->block_x, ctx->block_y, ctx->stream, e1, e2); break;
    case LBM_F16S: launch_step_f16(a, odd, epi, ctx->plain, ctx->block_x, ctx->block_y, ctx->stream, e1, e2); break;
    case LBM_BF16S: launch_step_bf16(a, odd, epi, ctx->plain, ctx->block_x, ctx->block_y, ctx->stream, e1, e2); break;
    default: launch_step_f16c(a, odd, epi, ctx->plain, ctx->block_x, ctx->block_y, ctx->stream, e1, e2); break;
    }
    if (e2) cudaEventRecord(e3, ctx->stream);
    ctx->launches += 1 + (a.n_edge > 0 || a.n_wall > 0 ? 1 : 0) + (a.face_x_hi == FACE_OUTFLOW ? 1 : 0) +
                     (a.n_qlinks > 0 ? 1 : 0);
}

// Outflow planes of the state before a step of parity `odd` (the convective
// outflow extrapolates from them after that step).
static void outflow_record(const lbm_ctx *c, const StepArgs &a, bool odd, cudaStream_t s)
{
    if (c->p.face_x_hi != LBM_FACE_OUTFLOW) return;
    switch (c->p.storage) {
    case LBM_F64: launch_outflow_record_f64(a, odd, s); break;
    case LBM_F32: launch_outflow_record_f32(a, odd, s); break;
    case LBM_F16S: launch_outflow_record_f16(a, odd, s); break;
    case LBM_BF16S: launch_outflow_record_bf16(a, odd, s); break;
    default: launch_outflow_record_f16c(a, odd, s); break;
    }
}

extern "C" lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps)
{
    if (!ctx || nsteps < 0) return ctx ? fail(ctx, LBM_ERR_ARG, "negative step count") : LBM_ERR_ARG;
    if (ctx->unstable) return fail(ctx, LBM_ERR_STATE, "state is unstable; steps refused");
    const lbm_params &p = ctx->p;
    const Layout &L = ctx->L;
    const StepArgs base = ctx->args();
    if (nsteps > 0) outflow_record(ctx, base, (ctx->t & 1) != 0, ctx->stream);
    for (int64_t k = 0; k < nsteps; ++k) {
        const int64_t t = ctx->t;
        StepArgs a = base;
        if (p.mean_every > 0 && t >= p.mean_start && t < p.mean_end && (t - p.mean_start) % p.mean_every == 0) {
            a.msum = ctx->at<double>(L.msum);
            ctx->msamples++;
        }
        int64_t snap_k = -1;
        if (p.snap_count > 0 && t >= p.snap_first && (t - p.snap_first) % p.snap_every == 0) {
            const int64_t kk = (t - p.snap_first) / p.snap_every;
            if (kk < p.snap_count) snap_k = kk;
        }
        float *slot = nullptr;
        if (snap_k >= 0) {
            slot = ctx->at<float>(L.snaps) + (size_t)snap_k * 4 * L.snap_cells;
            if (p.snap_halfres) {
                a.snap = ctx->at<float>(L.stage);
            } else {
                CK(cudaMemsetAsync(slot, 0, sizeof(float) * 4 * L.n, ctx->stream));
                a.snap = slot;
            }
            ctx->snap_taken[snap_k] = 1;
        }
        const bool rec_force = p.force_every > 0 && t % p.force_every == 0;
        if (rec_force) {
            if (ctx->force_rows_dev == ctx->force_cap) {
                lbm_status st = flush_forces(ctx);
                if (st != LBM_OK) return st;
            }
            a.fout = ctx->at<double>(L.force) + 3 * ctx->force_rows_dev;
            if (ctx->n_edge > 0) a.fpart = ctx->at<double>(L.fpart);
            else CK(cudaMemsetAsync(a.fout, 0, 3 * sizeof(double), ctx->stream));
            ctx->force_rows_dev++;
        }
        if (ctx->n_probes > 0 && t % ctx->probe_every == 0) {   // the state at t, before the step
            if (ctx->probe_rows_dev == ctx->probe_cap) {
                lbm_status st = flush_probes(ctx);
                if (st != LBM_OK) return st;
            }
            AuxArgs x;
            x.cells = ctx->probe_cells;
            x.count = ctx->n_probes;
            x.fout = ctx->probe_ring + 4 * ctx->n_probes * ctx->probe_rows_dev;
            launch_aux(p.storage, AUX_PROBE, base, (t & 1) != 0, x, ctx->stream);
            ctx->probe_rows_dev++;
            ctx->launches++;
        }
        if (ctx->plane_ring && t % ctx->plane_every == 0) {     // the state at t, before the step
            if (ctx->plane_rows_dev == ctx->plane_cap) {
                lbm_status st = flush_planes(ctx);
                if (st != LBM_OK) return st;
            }
            AuxArgs x;
            x.count = ctx->plane_z;
            x.fout = ctx->plane_ring + (size_t)4 * ctx->g.nx * ctx->g.ny * ctx->plane_rows_dev;
            launch_aux(p.storage, AUX_PLANE, base, (t & 1) != 0, x, ctx->stream);
            ctx->plane_rows_dev++;
            ctx->plane_steps.push_back(t);
            ctx->launches++;
        }
        step_launch(ctx, a, (t & 1) != 0, a.msum != nullptr || a.snap != nullptr);
        if (snap_k >= 0 && p.snap_halfres) {
            launch_halfres(a.snap, ctx->g.nx, ctx->g.ny, ctx->g.nz, true, slot, ctx->stream);
            ctx->launches++;
        }
        ctx->t = t + 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, LBM_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    return LBM_OK;
}

extern "C" lbm_status lbm_sync(lbm_ctx *ctx)
{
    if (!ctx) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    int st = 0;
    CK(cudaMemcpy(&st, ctx->base + ctx->L.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & STATUS_UNSTABLE) {
        ctx->unstable = true;
        return fail(ctx, LBM_ERR_UNSTABLE, "density left (0.5, 1.5) or became non-finite");
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// reads and writes
// ---------------------------------------------------------------------------
namespace {
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t b) { return cudaMalloc(&p, b ? b : 1); }
};
}  // namespace

// Run fn(dev_ptr) producing `bytes` of output at a device pointer, then place
// it into dst (device: directly; host: through a temporary).
template <class F>
static lbm_status produce(lbm_ctx *ctx, void *dst, size_t bytes, F fn)
{
    if (is_device_ptr(dst)) {
        fn(dst);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->stream));
        return LBM_OK;
    }
    DevBuf tmp;
    CK(tmp.alloc(bytes));
    fn(tmp.p);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dst, tmp.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_read_mean(lbm_ctx *ctx, int32_t dtype, int32_t halfres, void *dst, int64_t *samples)
{
    if (!ctx || !dst || (dtype != 0 && dtype != 1)) return ctx ? fail(ctx, LBM_ERR_ARG, "bad read_mean arguments") : LBM_ERR_ARG;
    if (ctx->p.mean_every <= 0) return fail(ctx, LBM_ERR_STATE, "time average not enabled");
    lbm_status st = lbm_sync(ctx);
    if (st != LBM_OK && st != LBM_ERR_UNSTABLE) return st;
    if (samples) *samples = ctx->msamples;
    const bool f32 = dtype == 1;
    const size_t es = f32 ? 4 : 8;
    const int64_t n = ctx->L.n, nh = ctx->L.n_half;
    const double inv = ctx->msamples > 0 ? 1.0 / (double)ctx->msamples : 0.0;
    const double *msum = ctx->at<double>(ctx->L.msum);
    if (!halfres)
        return produce(ctx, dst, 4 * es * n, [&](void *o) { launch_mean_out(msum, n, inv, f32, o, ctx->stream); });
    DevBuf full;
    CK(full.alloc(4 * es * n));
    launch_mean_out(msum, n, inv, f32, full.p, ctx->stream);
    return produce(ctx, dst, 4 * es * nh, [&](void *o) {
        launch_halfres(full.p, ctx->g.nx, ctx->g.ny, ctx->g.nz, f32, o, ctx->stream);
    });
}

// ---------------------------------------------------------------------------
// interpolated bounce-back: wall distances of obstacle links
// ---------------------------------------------------------------------------
extern "C" lbm_status lbm_set_wall_distances(lbm_ctx *ctx, int64_t n, const int64_t *cell, const int8_t *dir,
                                             const double *q)
{
    if (!ctx || n < 0 || (n > 0 && (!cell || !dir || !q))) return ctx ? fail(ctx, LBM_ERR_ARG, "bad wall-distance arguments") : LBM_ERR_ARG;
    if (ctx->in_batch) return fail(ctx, LBM_ERR_STATE, "set a batch member's wall distances with lbm_batch_set_wall_distances");
    const lbm_grid &g = ctx->g;
    const int64_t N = ctx->L.n;
    const lbm_params &p = ctx->p;
    // the cell (x, y, z), reached through periodic faces if needed, or -1
    auto wrap_cell = [&](int x, int y, int z) -> int64_t {
        if (x < 0 || x >= g.nx) {
            if (p.face_x_lo != LBM_FACE_PERIODIC) return -1;
            x = ((x % g.nx) + g.nx) % g.nx;
        }
        if (y < 0 || y >= g.ny) {
            if (p.face_y != LBM_FACE_PERIODIC) return -1;
            y = ((y % g.ny) + g.ny) % g.ny;
        }
        if (z < 0 || z >= g.nz) {
            if (p.face_z != LBM_FACE_PERIODIC) return -1;
            z = ((z % g.nz) + g.nz) % g.nz;
        }
        return (int64_t)x + (int64_t)g.nx * ((int64_t)y + (int64_t)g.ny * z);
    };
    // per link the cells whose class decides it: the fluid cell, the cell
    // behind the link (inside the grid), and the first and second cells
    // against the link (x1, x2); their flags are gathered on the device
    std::vector<int64_t> cand((size_t)4 * n, -1);
    for (int64_t k = 0; k < n; ++k) {
        const int64_t c = cell[k];
        const int j = dir[k];
        if (c < 0 || c >= N || j < 0 || j >= Q || j == 13 || !(q[k] > 0.0 && q[k] <= 1.0))
            return fail(ctx, LBM_ERR_ARG, "wall distance " + std::to_string(k) + ": cell, direction or q out of range");
        const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((int64_t)g.nx * g.ny));
        const int cx = cx_of(j), cy = cy_of(j), cz = cz_of(j);
        const int sx = x + cx, sy = y + cy, sz = z + cz;
        cand[4 * k] = c;
        if (sx >= 0 && sx < g.nx && sy >= 0 && sy < g.ny && sz >= 0 && sz < g.nz)
            cand[4 * k + 1] = (int64_t)sx + (int64_t)g.nx * ((int64_t)sy + (int64_t)g.ny * sz);
        cand[4 * k + 2] = wrap_cell(x - cx, y - cy, z - cz);
        cand[4 * k + 3] = wrap_cell(x - 2 * cx, y - 2 * cy, z - 2 * cz);
    }
    std::vector<uint8_t> fl((size_t)4 * n, 0);
    if (n > 0) {
        std::vector<int64_t> idx(cand);
        for (auto &v : idx) v = v < 0 ? 0 : v;
        int64_t *didx = nullptr;
        uint8_t *dfl = nullptr;
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMalloc(&didx, idx.size() * sizeof(int64_t)));
        if (cudaMalloc(&dfl, fl.size()) != cudaSuccess) {
            cudaFree(didx);
            return fail(ctx, LBM_ERR_CUDA, "wall-distance scratch allocation failed");
        }
        const bool ok = cudaMemcpy(didx, idx.data(), idx.size() * sizeof(int64_t), cudaMemcpyHostToDevice) == cudaSuccess &&
                        (launch_gather_flags(ctx->at<uint8_t>(ctx->L.flags), didx, (int64_t)idx.size(), dfl, nullptr),
                         cudaMemcpy(fl.data(), dfl, fl.size(), cudaMemcpyDeviceToHost) == cudaSuccess);
        cudaFree(didx);
        cudaFree(dfl);
        if (!ok) return fail(ctx, LBM_ERR_CUDA, std::string("wall-distance flag gather failed: ") +
                                                     cudaGetErrorString(cudaGetLastError()));
    }
    std::map<int64_t, std::pair<uint4, double>> recs;    // keyed by cell * 27 + j: the last entry wins
    for (int64_t k = 0; k < n; ++k) {
        const int64_t c = cell[k];
        const int j = dir[k];
        if ((fl[4 * k] & CELL_SOLID) || cand[4 * k + 1] < 0 || !(fl[4 * k + 1] & CELL_SOLID))
            return fail(ctx, LBM_ERR_ARG, "wall distance " + std::to_string(k) +
                                              ": not a link from a fluid cell into an obstacle cell");
        const int64_t x1 = cand[4 * k + 2], x2 = cand[4 * k + 3];
        const bool v1 = x1 >= 0 && !(fl[4 * k + 2] & CELL_SOLID);
        const bool v2 = v1 && x2 >= 0 && !(fl[4 * k + 3] & CELL_SOLID);
        const int mode = v1 ? (v2 ? 2 : 1) : 0;
        const int i = Q - 1 - j;                            // returning (pull) direction
        recs[c * Q + j] = {make_uint4((uint32_t)c, (uint32_t)(v1 ? x1 : c), (uint32_t)(v2 ? x2 : c),
                                      (uint32_t)(i | (mode << 8))), q[k]};
    }
    std::vector<uint4> L;
    std::vector<double> V;
    for (const auto &kv : recs)
        if ((kv.second.first.w >> 8) != 0) {               // mode 0: halfway bounce-back, nothing to do
            L.push_back(kv.second.first);
            V.push_back(kv.second.second);
        }
    cudaFree(ctx->qlinks); cudaFree(ctx->qval); cudaFree(ctx->qpart); cudaFree(ctx->qcount);
    ctx->qlinks = nullptr; ctx->qval = nullptr; ctx->qpart = nullptr; ctx->qcount = nullptr;
    ctx->n_qlinks = 0;
    if (L.empty()) return LBM_OK;
    const int64_t m = (int64_t)L.size(), nb = (m + EDGE_BLOCK - 1) / EDGE_BLOCK;
    CK(cudaMalloc(&ctx->qlinks, m * sizeof(uint4)));
    CK(cudaMalloc(&ctx->qval, m * sizeof(double)));
    CK(cudaMalloc(&ctx->qpart, 3 * sizeof(double) * nb));
    CK(cudaMalloc(&ctx->qcount, sizeof(unsigned)));
    CK(cudaMemcpy(ctx->qlinks, L.data(), m * sizeof(uint4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->qval, V.data(), m * sizeof(double), cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->qcount, 0, sizeof(unsigned)));
    ctx->n_qlinks = m;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// probes
// ---------------------------------------------------------------------------
extern "C" lbm_status lbm_set_probes(lbm_ctx *ctx, int64_t n, const int64_t *cells, int64_t every, int64_t capacity)
{
    if (!ctx || n < 0 || (n > 0 && (!cells || every < 1 || capacity < 1)))
        return ctx ? fail(ctx, LBM_ERR_ARG, "bad probe arguments") : LBM_ERR_ARG;
    if (ctx->in_batch) return fail(ctx, LBM_ERR_STATE, "probes are not supported on batch members");
    for (int64_t k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= ctx->L.n) return fail(ctx, LBM_ERR_ARG, "probe cell out of range");
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->probe_cells);
    cudaFree(ctx->probe_ring);
    ctx->probe_cells = nullptr;
    ctx->probe_ring = nullptr;
    ctx->n_probes = 0;
    ctx->probe_rows_dev = 0;
    ctx->probe_host.clear();
    if (n == 0) return LBM_OK;
    CK(cudaMalloc(&ctx->probe_cells, sizeof(int64_t) * n));
    CK(cudaMalloc(&ctx->probe_ring, sizeof(float) * 4 * n * capacity));
    CK(cudaMemcpy(ctx->probe_cells, cells, sizeof(int64_t) * n, cudaMemcpyHostToDevice));
    ctx->n_probes = n;
    ctx->probe_every = every;
    ctx->probe_cap = capacity;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// monitor plane (Sec. 2: 2D snapshots of the centre x-y plane)
// ---------------------------------------------------------------------------
extern "C" lbm_status lbm_set_plane_monitor(lbm_ctx *ctx, int32_t z, int64_t every, int64_t capacity)
{
    if (!ctx) return LBM_ERR_ARG;
    if (ctx->in_batch) return fail(ctx, LBM_ERR_STATE, "the monitor plane is not supported on batch members");
    if (every < 0 || (every > 0 && capacity < 1)) return fail(ctx, LBM_ERR_ARG, "bad monitor-plane arguments");
    const int zz = z < 0 ? ctx->g.nz / 2 : z;
    if (zz >= ctx->g.nz) return fail(ctx, LBM_ERR_ARG, "monitor plane z out of range");
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->plane_ring);
    ctx->plane_ring = nullptr;
    ctx->plane_rows_dev = 0;
    ctx->plane_host.clear();
    ctx->plane_steps.clear();
    if (every == 0) return LBM_OK;
    CK(cudaMalloc(&ctx->plane_ring, sizeof(float) * 4 * (size_t)ctx->g.nx * ctx->g.ny * capacity));
    ctx->plane_z = zz;
    ctx->plane_every = every;
    ctx->plane_cap = capacity;
    return LBM_OK;
}

extern "C" lbm_status lbm_read_plane_monitor(lbm_ctx *ctx, float *dst, int64_t max_planes, int64_t *n_planes,
                                             int64_t *steps)
{
    if (!ctx || max_planes < 0 || (max_planes > 0 && !dst))
        return ctx ? fail(ctx, LBM_ERR_ARG, "bad monitor-plane read arguments") : LBM_ERR_ARG;
    lbm_status st = flush_planes(ctx);
    if (st != LBM_OK) return st;
    const int64_t per = 4 * (int64_t)ctx->g.nx * ctx->g.ny;
    const int64_t rows = (int64_t)ctx->plane_steps.size();
    if (n_planes) *n_planes = rows;
    const int64_t m = std::min(rows, max_planes);
    if (m > 0) {
        if (is_device_ptr(dst)) CK(cudaMemcpy(dst, ctx->plane_host.data(), sizeof(float) * per * m, cudaMemcpyHostToDevice));
        else std::memcpy(dst, ctx->plane_host.data(), sizeof(float) * per * m);
        if (steps) std::memcpy(steps, ctx->plane_steps.data(), sizeof(int64_t) * m);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_read_probes(lbm_ctx *ctx, float *dst, int64_t max_rows, int64_t *n_rows)
{
    if (!ctx || max_rows < 0 || (max_rows > 0 && !dst)) return LBM_ERR_ARG;
    lbm_status st = flush_probes(ctx);
    if (st != LBM_OK) return st;
    const int64_t per = 4 * ctx->n_probes;
    const int64_t rows = per > 0 ? (int64_t)ctx->probe_host.size() / per : 0;
    if (n_rows) *n_rows = rows;
    const int64_t m = std::min(rows, max_rows);
    if (m > 0) {
        if (is_device_ptr(dst)) CK(cudaMemcpy(dst, ctx->probe_host.data(), sizeof(float) * per * m, cudaMemcpyHostToDevice));
        else std::memcpy(dst, ctx->probe_host.data(), sizeof(float) * per * m);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_read_stats(lbm_ctx *ctx, int32_t dtype, void *dst, int64_t *samples)
{
    if (!ctx || !dst || (dtype != 0 && dtype != 1)) return ctx ? fail(ctx, LBM_ERR_ARG, "bad read_stats arguments") : LBM_ERR_ARG;
    if (ctx->p.mean_every <= 0 || !ctx->p.stats) return fail(ctx, LBM_ERR_STATE, "turbulence statistics not enabled");
    lbm_status st = lbm_sync(ctx);
    if (st != LBM_OK && st != LBM_ERR_UNSTABLE) return st;
    if (samples) *samples = ctx->msamples;
    const bool f32 = dtype == 1;
    const int64_t n = ctx->L.n;
    const double inv = ctx->msamples > 0 ? 1.0 / (double)ctx->msamples : 0.0;
    const double *msum = ctx->at<double>(ctx->L.msum);
    return produce(ctx, dst, 6 * (f32 ? 4 : 8) * n, [&](void *o) { launch_stats_out(msum, n, inv, f32, o, ctx->stream); });
}

extern "C" lbm_status lbm_read_snapshot(lbm_ctx *ctx, int32_t k, float *dst)
{
    if (!ctx || !dst) return LBM_ERR_ARG;
    if (k < 0 || k >= ctx->p.snap_count) return fail(ctx, LBM_ERR_ARG, "snapshot index out of range");
    if (!ctx->snap_taken[k]) return fail(ctx, LBM_ERR_STATE, "snapshot not taken yet");
    CK(cudaStreamSynchronize(ctx->stream));
    const size_t bytes = sizeof(float) * 4 * ctx->L.snap_cells;
    CK(cudaMemcpyAsync(dst, ctx->at<float>(ctx->L.snaps) + (size_t)k * 4 * ctx->L.snap_cells, bytes,
                       cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_read_macros(lbm_ctx *ctx, double *rho, double *u)
{
    if (!ctx || !rho || !u) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t n = ctx->L.n;
    DevBuf br, bu;
    CK(br.alloc(8 * n));
    CK(bu.alloc(24 * n));
    AuxArgs x;
    x.out = (double *)br.p;
    x.out2 = (double *)bu.p;
    launch_aux(ctx->p.storage, AUX_MACROS, ctx->args(), ctx->t & 1, x, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(rho, br.p, 8 * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(u, bu.p, 24 * n, cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_read_forces(lbm_ctx *ctx, double *dst, int64_t max_rows, int64_t *n_rows)
{
    if (!ctx || max_rows < 0 || (max_rows > 0 && !dst)) return LBM_ERR_ARG;
    lbm_status st = flush_forces(ctx);
    if (st != LBM_OK) return st;
    const int64_t rows = (int64_t)ctx->force_host.size() / 3;
    if (n_rows) *n_rows = rows;
    const int64_t m = std::min(rows, max_rows);
    std::vector<double> out(3 * m);
    for (int64_t r = 0; r < m; ++r)
        for (int d = 0; d < 3; ++d) out[3 * r + d] = ctx->force_host[3 * r + d] + ctx->force_w[d];
    if (m > 0) {
        if (is_device_ptr(dst)) CK(cudaMemcpy(dst, out.data(), sizeof(double) * 3 * m, cudaMemcpyHostToDevice));
        else std::memcpy(dst, out.data(), sizeof(double) * 3 * m);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_get_pdfs(lbm_ctx *ctx, double *dst)
{
    if (!ctx || !dst) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t n = ctx->L.n;
    return produce(ctx, dst, sizeof(double) * Q * n, [&](void *o) {
        AuxArgs x;
        x.count = n; x.out = (double *)o; x.si = n; x.sc = 1;
        launch_aux(ctx->p.storage, AUX_GATHER, ctx->args(), ctx->t & 1, x, ctx->stream);
    });
}

extern "C" lbm_status lbm_get_cells(lbm_ctx *ctx, int64_t count, const int64_t *cells, double *dst)
{
    if (!ctx || count < 0 || (count > 0 && (!cells || !dst))) return LBM_ERR_ARG;
    if (count == 0) return LBM_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    DevBuf dc;
    const int64_t *dcells = cells;
    if (!is_device_ptr(cells)) {
        for (int64_t k = 0; k < count; ++k)
            if (cells[k] < 0 || cells[k] >= ctx->L.n) return fail(ctx, LBM_ERR_ARG, "cell index out of range");
        CK(dc.alloc(8 * count));
        CK(cudaMemcpyAsync(dc.p, cells, 8 * count, cudaMemcpyHostToDevice, ctx->stream));
        dcells = (const int64_t *)dc.p;
    }
    return produce(ctx, dst, sizeof(double) * Q * count, [&](void *o) {
        AuxArgs x;
        x.cells = dcells; x.count = count; x.out = (double *)o; x.si = 1; x.sc = Q;
        launch_aux(ctx->p.storage, AUX_GATHER, ctx->args(), ctx->t & 1, x, ctx->stream);
    });
}

extern "C" lbm_status lbm_init_equilibrium(lbm_ctx *ctx, const float *fields)
{
    if (!ctx || !fields) return LBM_ERR_ARG;
    if (ctx->t & 1) return fail(ctx, LBM_ERR_STATE, "init_equilibrium needs an even time step");
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t n = ctx->L.n;
    DevBuf tmp;
    const float *dsrc = fields;
    if (!is_device_ptr(fields) || ((uintptr_t)fields & 15) != 0) {
        CK(tmp.alloc(sizeof(float) * 4 * n));
        CK(cudaMemcpyAsync(tmp.p, fields, sizeof(float) * 4 * n, cudaMemcpyDefault, ctx->stream));
        dsrc = (const float *)tmp.p;
    }
    AuxArgs x;
    x.fsrc = dsrc;
    launch_aux(ctx->p.storage, AUX_EQUILIBRIUM, ctx->args(), false, x, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_set_pdfs(lbm_ctx *ctx, const double *src)
{
    if (!ctx || !src) return LBM_ERR_ARG;
    if (ctx->t & 1) return fail(ctx, LBM_ERR_STATE, "set_pdfs needs an even time step");
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t n = ctx->L.n;
    DevBuf tmp;
    const double *dsrc = src;
    if (!is_device_ptr(src)) {
        CK(tmp.alloc(sizeof(double) * Q * n));
        CK(cudaMemcpyAsync(tmp.p, src, sizeof(double) * Q * n, cudaMemcpyHostToDevice, ctx->stream));
        dsrc = (const double *)tmp.p;
    }
    AuxArgs x;
    x.src = dsrc;
    launch_aux(ctx->p.storage, AUX_SET, ctx->args(), false, x, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

extern "C" lbm_status lbm_init_noise(lbm_ctx *ctx, uint64_t seed, double amplitude)
{
    if (!ctx) return LBM_ERR_ARG;
    if (ctx->t & 1) return fail(ctx, LBM_ERR_STATE, "init_noise needs an even time step");
    AuxArgs x;
    x.seed = seed;
    x.amp = amplitude;
    launch_aux(ctx->p.storage, AUX_NOISE, ctx->args(), false, x, ctx->stream);
    CK(cudaGetLastError());
    return LBM_OK;
}

extern "C" lbm_status lbm_totals(lbm_ctx *ctx, double out[4])
{
    if (!ctx || !out) return LBM_ERR_ARG;
    AuxArgs x;
    x.partials = ctx->at<double>(ctx->L.tpart);
    x.nblocks = ctx->L.tot_blocks;
    x.out = ctx->at<double>(ctx->L.tout);
    launch_aux(ctx->p.storage, AUX_TOTALS, ctx->args(), ctx->t & 1, x, ctx->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, x.out, 4 * sizeof(double), cudaMemcpyDefault, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// checkpoints
// ---------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, storage, nx, ny, nz, pad;
    int64_t t, msamples, force_rows, n_edge, snap_count;
};
}  // namespace

extern "C" lbm_status lbm_save(lbm_ctx *ctx, const char *path)
{
    if (!ctx || !path) return LBM_ERR_ARG;
    lbm_status st = flush_forces(ctx);
    if (st != LBM_OK) return st;
    const Layout &L = ctx->L;
    const size_t es = storage_bytes(ctx->p.storage);
    const size_t pdf_bytes = (size_t)Q * L.slot * es;
    const size_t ub_bytes = (size_t)3 * ctx->g.ny * ctx->g.nz * (ctx->p.storage == LBM_F64 ? 8 : 4);
    const size_t ms_bytes = msum_bytes(ctx->p, L.n);
    std::vector<char> buf(pdf_bytes + ub_bytes + ms_bytes);
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(buf.data(), ctx->base + L.pdf, pdf_bytes, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(buf.data() + pdf_bytes, ctx->base + L.ub, ub_bytes, cudaMemcpyDeviceToHost));
    if (ms_bytes) CK(cudaMemcpy(buf.data() + pdf_bytes + ub_bytes, ctx->base + L.msum, ms_bytes, cudaMemcpyDeviceToHost));
    CkptHeader h{};
    std::memcpy(h.magic, "GBLBMCK1", 8);
    h.version = 1; h.storage = ctx->p.storage; h.nx = ctx->g.nx; h.ny = ctx->g.ny; h.nz = ctx->g.nz;
    h.t = ctx->t; h.msamples = ctx->msamples; h.force_rows = (int64_t)ctx->force_host.size() / 3;
    h.n_edge = ctx->n_edge; h.snap_count = ctx->p.snap_count;
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return fail(ctx, LBM_ERR_IO, std::string("cannot open ") + path);
    bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1;
    ok = ok && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    if (h.force_rows) ok = ok && std::fwrite(ctx->force_host.data(), sizeof(double), ctx->force_host.size(), fp) == ctx->force_host.size();
    if (h.snap_count) ok = ok && std::fwrite(ctx->snap_taken.data(), 1, ctx->snap_taken.size(), fp) == ctx->snap_taken.size();
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(ctx, LBM_ERR_IO, "checkpoint write failed");
}

extern "C" lbm_status lbm_load(lbm_ctx *ctx, const char *path)
{
    if (!ctx || !path) return LBM_ERR_ARG;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return fail(ctx, LBM_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h{};
    if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, "GBLBMCK1", 8) != 0 ||
        h.storage != ctx->p.storage || h.nx != ctx->g.nx || h.ny != ctx->g.ny || h.nz != ctx->g.nz ||
        h.n_edge != ctx->n_edge || h.snap_count != ctx->p.snap_count) {
        std::fclose(fp);
        return fail(ctx, LBM_ERR_IO, "checkpoint does not match this context");
    }
    const Layout &L = ctx->L;
    const size_t es = storage_bytes(ctx->p.storage);
    const size_t pdf_bytes = (size_t)Q * L.slot * es;
    const size_t ub_bytes = (size_t)3 * ctx->g.ny * ctx->g.nz * (ctx->p.storage == LBM_F64 ? 8 : 4);
    const size_t ms_bytes = msum_bytes(ctx->p, L.n);
    std::vector<char> buf(pdf_bytes + ub_bytes + ms_bytes);
    std::vector<double> frows(3 * h.force_rows);
    std::vector<char> taken(h.snap_count);
    bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    if (h.force_rows) ok = ok && std::fread(frows.data(), sizeof(double), frows.size(), fp) == frows.size();
    if (h.snap_count) ok = ok && std::fread(taken.data(), 1, taken.size(), fp) == taken.size();
    std::fclose(fp);
    if (!ok) return fail(ctx, LBM_ERR_IO, "checkpoint truncated");
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->base + L.pdf, buf.data(), pdf_bytes, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->base + L.ub, buf.data() + pdf_bytes, ub_bytes, cudaMemcpyHostToDevice));
    if (ms_bytes) CK(cudaMemcpy(ctx->base + L.msum, buf.data() + pdf_bytes + ub_bytes, ms_bytes, cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->base + L.status, 0, sizeof(int)));
    ctx->t = h.t;
    ctx->msamples = h.msamples;
    ctx->force_host = frows;
    ctx->force_rows_dev = 0;
    ctx->snap_taken = taken;
    ctx->unstable = false;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_info(const lbm_ctx *ctx, lbm_info *out)
{
    if (!ctx || !out) return LBM_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->cells = ctx->L.n;
    out->fluid_cells = ctx->n_fluid;
    out->edge_cells = ctx->n_edge;
    out->bulk_cells = ctx->n_bulk;
    out->interior_cells = ctx->n_bulk;
    out->wall_cells = ctx->n_wall;
    out->launches = ctx->launches;
    out->workspace_bytes = ctx->L.total;
    out->storage = ctx->p.storage;
    out->block_x = ctx->block_x;
    out->omega1 = ctx->w1;
    return LBM_OK;
}

extern "C" lbm_status lbm_timing(lbm_ctx *ctx, int32_t enable)
{
    if (!ctx) return LBM_ERR_ARG;
    ctx->timing = enable != 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_timing_read(lbm_ctx *ctx, lbm_timing_report *out, int32_t reset)
{
    if (!ctx || !out) return LBM_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    std::memset(out, 0, sizeof(*out));
    for (size_t k = 0; k < ctx->ev_kind.size(); ++k) {
        float a = 0.f, b = 0.f, c = 0.f;
        CK(cudaEventElapsedTime(&a, ctx->ev_pool[4 * k], ctx->ev_pool[4 * k + 1]));
        CK(cudaEventElapsedTime(&b, ctx->ev_pool[4 * k + 1], ctx->ev_pool[4 * k + 2]));
        CK(cudaEventElapsedTime(&c, ctx->ev_pool[4 * k + 2], ctx->ev_pool[4 * k + 3]));
        const int kind = ctx->ev_kind[k];
        out->bulk_ms[kind] += a;
        out->bulk_n[kind] += 1;
        out->rowend_ms += b;
        out->edge_ms += c;
    }
    out->steps = (int64_t)ctx->ev_kind.size();
    if (reset) {
        ctx->ev_kind.clear();
        ctx->ev_used = 0;
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// reset to rest
// ---------------------------------------------------------------------------
extern "C" lbm_status lbm_reset(lbm_ctx *ctx)
{
    if (!ctx) return LBM_ERR_ARG;
    const Layout &L = ctx->L;
    const lbm_params &p = ctx->p;
    cudaStream_t s = ctx->stream;
    CK(cudaStreamSynchronize(s));
    CK(cudaMemsetAsync(ctx->base + L.pdf, 0, (size_t)Q * L.slot * storage_bytes(p.storage), s));
    CK(cudaMemsetAsync(ctx->base + L.ub, 0, (size_t)3 * ctx->g.ny * ctx->g.nz * (p.storage == LBM_F64 ? 8 : 4), s));
    if (p.mean_every > 0) CK(cudaMemsetAsync(ctx->base + L.msum, 0, msum_bytes(p, L.n), s));
    if (p.force_every > 0) CK(cudaMemsetAsync(ctx->base + L.force, 0, (size_t)ctx->force_cap * 3 * 8, s));
    CK(cudaMemsetAsync(ctx->base + L.fcount, 0, sizeof(unsigned), s));
    CK(cudaMemsetAsync(ctx->base + L.status, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    ctx->t = 0;
    ctx->msamples = 0;
    ctx->force_host.clear();
    ctx->force_rows_dev = 0;
    ctx->probe_host.clear();
    ctx->probe_rows_dev = 0;
    ctx->plane_host.clear();
    ctx->plane_steps.clear();
    ctx->plane_rows_dev = 0;
    std::fill(ctx->snap_taken.begin(), ctx->snap_taken.end(), 0);
    ctx->unstable = false;
    ctx->ev_kind.clear();
    ctx->ev_used = 0;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// autotuner cache: a flat JSON object {"key": [block_x, block_y, ms], ...}
// ---------------------------------------------------------------------------
namespace {
const int TUNE_CAND[][2] = {{64, 1}, {128, 1}, {256, 1}, {64, 2}, {128, 2}, {32, 4}, {32, 8}};
constexpr int N_TUNE_CAND = 7;

std::string tune_key(const std::string &what)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    std::string name = cudaGetDeviceProperties(&pr, dev) == cudaSuccess ? pr.name : "gpu";
    for (char &ch : name)
        if (ch == '"' || ch == ' ') ch = '_';
    return name + "|" + what;
}

bool tune_lookup(const std::string &key, int *bx, int *by, double *ms)
{
    const char *path = std::getenv("LBM_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return false;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof buf, fp)) > 0) text.append(buf, r);
    std::fclose(fp);
    const std::string pat = "\"" + key + "\": [";
    const size_t pos = text.find(pat);
    if (pos == std::string::npos) return false;
    return std::sscanf(text.c_str() + pos + pat.size(), "%d, %d, %lf", bx, by, ms) == 3;
}

void tune_store(const std::string &key, int bx, int by, double ms)
{
    const char *path = std::getenv("LBM_AUTOTUNE_CACHE");
    if (!path) return;
    std::vector<std::string> entries;
    if (FILE *fp = std::fopen(path, "rb")) {
        std::string text;
        char buf[4096];
        size_t r;
        while ((r = std::fread(buf, 1, sizeof buf, fp)) > 0) text.append(buf, r);
        std::fclose(fp);
        size_t pos = 0;
        while ((pos = text.find('"', pos)) != std::string::npos) {
            const size_t end = text.find(']', pos);
            if (end == std::string::npos) break;
            std::string e = text.substr(pos, end - pos + 1);
            if (e.compare(0, key.size() + 2, "\"" + key + "\"") != 0) entries.push_back(e);
            pos = end + 1;
        }
    }
    char line[512];
    std::snprintf(line, sizeof line, "\"%s\": [%d, %d, %.6f]", key.c_str(), bx, by, ms);
    entries.push_back(line);
    const std::string tmp = std::string(path) + ".tmp";
    if (FILE *fp = std::fopen(tmp.c_str(), "wb")) {
        std::fputs("{\n", fp);
        for (size_t k = 0; k < entries.size(); ++k)
            std::fprintf(fp, "  %s%s\n", entries[k].c_str(), k + 1 < entries.size() ? "," : "");
        std::fputs("}\n", fp);
        std::fclose(fp);
        std::rename(tmp.c_str(), path);
    }
}
}  // namespace

extern "C" lbm_status lbm_autotune(lbm_ctx *ctx, int32_t trials, int32_t *best_bx, int32_t *best_by, double *best_ms)
{
    if (!ctx || trials < 2) return ctx ? fail(ctx, LBM_ERR_ARG, "autotune needs trials >= 2") : LBM_ERR_ARG;
    char what[256];
    std::snprintf(what, sizeof what, "ctx|s%d|p%d|%dx%dx%d", ctx->p.storage, (int)ctx->plain, ctx->g.nx, ctx->g.ny,
                  ctx->g.nz);
    const std::string key = tune_key(what);
    int bx = 0, by = 0;
    double ms = 0;
    if (!tune_lookup(key, &bx, &by, &ms)) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        double best = 1e300;
        const int64_t nt = trials + (trials & 1);
        for (int c = 0; c < N_TUNE_CAND; ++c) {
            ctx->block_x = TUNE_CAND[c][0];
            ctx->block_y = TUNE_CAND[c][1];
            lbm_status st = lbm_step(ctx, 2);        // warm-up
            if (st == LBM_OK) {
                cudaEventRecord(e0, ctx->stream);
                st = lbm_step(ctx, nt);
                cudaEventRecord(e1, ctx->stream);
            }
            if (st != LBM_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st != LBM_OK ? st : fail(ctx, LBM_ERR_CUDA, "autotune timing failed");
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t / nt < best) { best = t / nt; bx = ctx->block_x; by = ctx->block_y; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ms = best;
        tune_store(key, bx, by, ms);
    }
    ctx->block_x = bx;
    ctx->block_y = by;
    if (best_bx) *best_bx = bx;
    if (best_by) *best_by = by;
    if (best_ms) *best_ms = ms;
    return lbm_reset(ctx);
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct lbm_batch {
    std::vector<lbm_ctx *> members;
    std::vector<int64_t> t_end;
    int64_t t = 0;
    int64_t chunk = 2;
    int64_t mean_every = 0;
    int storage = LBM_F32;
    bool plain = true;
    int block_x = 128, block_y = 1;
    cudaStream_t user = nullptr, own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    BatchMember *d_mem = nullptr;
    int64_t *d_bbegin = nullptr, *d_ebegin = nullptr, *d_qbegin = nullptr, *d_wbegin = nullptr, *d_t = nullptr;
    std::vector<int> live;              // members in the current table
    BatchLaunch launch{};
    cudaGraphExec_t graph = nullptr;
    int64_t captures = 0, graph_launches = 0, kernel_launches = 0, updates = 0;
    std::string err;
};

#define BCK(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            g_err = b->err;                                                              \
            return LBM_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

static lbm_status batch_fail(lbm_batch *b, lbm_status s, const std::string &m)
{
    if (b) b->err = m;
    g_err = m;
    return s;
}

extern "C" lbm_status lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_ERR_ARG;
    if (b->own) cudaStreamSynchronize(b->own);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_mem) cudaFree(b->d_mem);
    if (b->d_bbegin) cudaFree(b->d_bbegin);
    if (b->d_ebegin) cudaFree(b->d_ebegin);
    if (b->d_qbegin) cudaFree(b->d_qbegin);
    if (b->d_wbegin) cudaFree(b->d_wbegin);
    if (b->d_t) cudaFree(b->d_t);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->own) cudaStreamDestroy(b->own);
    for (lbm_ctx *c : b->members) lbm_destroy(c);
    delete b;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_create(int32_t n, const lbm_grid *grids, const uint8_t *const *masks,
                                       const lbm_params *params, void *cuda_stream, lbm_batch **out)
{
    if (!out || n < 1 || !grids || !params) return batch_fail(nullptr, LBM_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    const lbm_params &p0 = params[0];
    int64_t me = 0;
    for (int g = 0; g < n; ++g) {
        const lbm_params &p = params[g];
        if (p.storage != p0.storage) return batch_fail(nullptr, LBM_ERR_ARG, "batch members need one storage");
        if ((p.omega_higher == 1.0 && !p.param4) != (p0.omega_higher == 1.0 && !p0.param4))
            return batch_fail(nullptr, LBM_ERR_ARG,
                              "batch members need the same collision kind (plain: omega_higher == 1, no param4)");
        if (p.snap_count > 0) return batch_fail(nullptr, LBM_ERR_ARG, "batch members take no snapshots");
        if (p.mean_every > 0) {
            if (me && p.mean_every != me) return batch_fail(nullptr, LBM_ERR_ARG, "batch members need one mean_every");
            me = p.mean_every;
        }
    }
    if (me % 2 != 0) return batch_fail(nullptr, LBM_ERR_ARG, "mean_every must be even in a batch");
    for (int g = 0; g < n; ++g)
        if (params[g].mean_every > 0 && params[g].mean_start % me != 0)
            return batch_fail(nullptr, LBM_ERR_ARG, "mean_start must be a multiple of mean_every in a batch");
    lbm_batch *b = new lbm_batch();
    b->user = static_cast<cudaStream_t>(cuda_stream);
    b->mean_every = me;
    b->chunk = me > 0 ? me : 2;
    b->storage = p0.storage;
    b->plain = p0.omega_higher == 1.0 && !p0.param4;
    b->block_x = p0.block_x ? p0.block_x : 128;
    b->block_y = p0.block_y ? p0.block_y : 1;
    for (int g = 0; g < n; ++g) {
        lbm_ctx *c = nullptr;
        // the inlet/outlet cells ride in the batched bulk kernel's face warps
        // (coalesced with their rows) unless a member asks for the
        // boundary-cell records (xface_edge): as records every one of their
        // 54 accesses is a sector of its own (the plane is strided by nx),
        // which took a third of a step of the 32-channel batch
        lbm_status st = lbm_create(&grids[g], masks ? masks[g] : nullptr, &params[g], cuda_stream, &c);
        if (st != LBM_OK) {
            const std::string m = "member " + std::to_string(g) + ": " + g_err;
            lbm_batch_destroy(b);
            return batch_fail(nullptr, st, m);
        }
        c->in_batch = true;
        b->members.push_back(c);
        b->t_end.push_back(INT64_MAX / 4);
    }
    lbm_status st = LBM_OK;
    if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&b->d_mem, sizeof(BatchMember) * n) != cudaSuccess ||
        cudaMalloc(&b->d_bbegin, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_ebegin, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_qbegin, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_wbegin, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_t, sizeof(int64_t)) != cudaSuccess ||
        cudaMemset(b->d_t, 0, sizeof(int64_t)) != cudaSuccess)
        st = LBM_ERR_CUDA;
    if (st != LBM_OK) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return batch_fail(nullptr, st, "batch device set-up failed");
    }
    *out = b;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_set_wall_distances(lbm_batch *b, int32_t g, int64_t n, const int64_t *cell,
                                                   const int8_t *dir, const double *q)
{
    if (!b || g < 0 || g >= (int32_t)b->members.size()) return LBM_ERR_ARG;
    lbm_ctx *c = b->members[g];
    c->in_batch = false;
    const lbm_status st = lbm_set_wall_distances(c, n, cell, dir, q);
    c->in_batch = true;
    if (st != LBM_OK) return batch_fail(b, st, "member " + std::to_string(g) + ": " + c->err);
    if (b->graph) {                                     // the member table changes: capture again
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_member(lbm_batch *b, int32_t g, lbm_ctx **ctx)
{
    if (!b || !ctx || g < 0 || g >= (int32_t)b->members.size()) return LBM_ERR_ARG;
    *ctx = b->members[g];
    return LBM_OK;
}

static int64_t round_chunk(const lbm_batch *b, int64_t v) { return (v + b->chunk - 1) / b->chunk * b->chunk; }

extern "C" lbm_status lbm_batch_set_end(lbm_batch *b, const int64_t *t_end)
{
    if (!b || !t_end) return LBM_ERR_ARG;
    for (size_t g = 0; g < b->members.size(); ++g) {
        if (t_end[g] < 0) return batch_fail(b, LBM_ERR_ARG, "negative end step");
        const lbm_ctx *c = b->members[g];
        // an end at or before the batch time retires the member now
        const int64_t te = t_end[g] <= b->t ? std::min(b->t, b->t_end[g]) : round_chunk(b, t_end[g]);
        if (c->p.force_every > 0 && te / c->p.force_every + 1 > c->force_cap)
            return batch_fail(b, LBM_ERR_ARG, "force_capacity of member " + std::to_string(g) + " is too small");
        b->t_end[g] = te;
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_set_flowthroughs(lbm_batch *b, double n_ft)
{
    if (!b || !(n_ft >= 0)) return LBM_ERR_ARG;
    std::vector<int64_t> te(b->members.size());
    for (size_t g = 0; g < b->members.size(); ++g) {
        const lbm_ctx *c = b->members[g];
        if (!(c->p.u_in > 0)) return batch_fail(b, LBM_ERR_ARG, "flow-through time needs u_in > 0");
        const double steps = n_ft * c->g.nx / c->p.u_in;
        te[g] = (int64_t)std::ceil(steps * (1.0 - 1e-12));   // integral counts stay integral
    }
    return lbm_batch_set_end(b, te.data());
}

// Build the member table of the live members and capture one chunk as a graph.
static lbm_status batch_rebuild(lbm_batch *b, const std::vector<int> &live)
{
    std::vector<BatchMember> mem(live.size());
    std::vector<int64_t> bb(live.size() + 1, 0), eb(live.size() + 1, 0), qb(live.size() + 1, 0),
        wb(live.size() + 1, 0);
    for (size_t k = 0; k < live.size(); ++k) {
        lbm_ctx *c = b->members[live[k]];
        BatchMember &M = mem[k];
        std::memset(&M, 0, sizeof(M));
        M.a = c->args();
        M.a.fpart = c->at<double>(c->L.fpart);
        M.msum = c->p.mean_every > 0 ? c->at<double>(c->L.msum) : nullptr;
        M.mean_start = c->p.mean_start;
        M.mean_end = c->p.mean_end;
        M.mean_every = c->p.mean_every;
        M.force = c->p.force_every > 0 ? c->at<double>(c->L.force) : nullptr;
        M.force_every = c->p.force_every > 0 ? c->p.force_every : 1;
        M.gx = (c->g.nx + b->block_x - 1) / b->block_x;
        M.gy = (c->g.ny + b->block_y - 1) / b->block_y;
        bb[k + 1] = bb[k] + (int64_t)M.gx * M.gy * c->g.nz;
        eb[k + 1] = eb[k] + (c->n_edge + EDGE_BLOCK - 1) / EDGE_BLOCK;
        qb[k + 1] = qb[k] + (c->n_qlinks + EDGE_BLOCK - 1) / EDGE_BLOCK;
        M.wx = (c->g.nx + WALL_BLOCK - 1) / WALL_BLOCK;
        wb[k + 1] = wb[k] + (c->n_wall > 0 ? (int64_t)M.wx * wall_rows(c->g.ny, c->g.nz) : 0);
    }
    if (bb.back() >= (int64_t(1) << 31) || eb.back() >= (int64_t(1) << 31) || wb.back() >= (int64_t(1) << 31))
        return batch_fail(b, LBM_ERR_ARG, "batch too large for one launch");
    BCK(cudaMemcpyAsync(b->d_mem, mem.data(), sizeof(BatchMember) * mem.size(), cudaMemcpyHostToDevice, b->own));
    BCK(cudaMemcpyAsync(b->d_bbegin, bb.data(), sizeof(int64_t) * bb.size(), cudaMemcpyHostToDevice, b->own));
    BCK(cudaMemcpyAsync(b->d_ebegin, eb.data(), sizeof(int64_t) * eb.size(), cudaMemcpyHostToDevice, b->own));
    BCK(cudaStreamSynchronize(b->own));
    int out_chunks = 0;
    for (int g : live) {
        const lbm_ctx *c = b->members[g];
        if (c->p.face_x_hi == LBM_FACE_OUTFLOW)
            out_chunks = std::max<int>(out_chunks, (int)std::min<int64_t>((9 * (int64_t)c->g.ny * c->g.nz + 255) / 256, 256));
    }
    BCK(cudaMemcpyAsync(b->d_qbegin, qb.data(), sizeof(int64_t) * qb.size(), cudaMemcpyHostToDevice, b->own));
    BCK(cudaMemcpyAsync(b->d_wbegin, wb.data(), sizeof(int64_t) * wb.size(), cudaMemcpyHostToDevice, b->own));
    BCK(cudaStreamSynchronize(b->own));
    b->launch = BatchLaunch{b->d_mem, b->d_bbegin, b->d_ebegin, (int)live.size(), bb.back(), eb.back(), b->d_t,
                            b->block_x, b->block_y, out_chunks, b->d_qbegin, qb.back(), b->d_wbegin, wb.back()};
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t graph;
    BCK(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
    for (int64_t k = 0; k < b->chunk; ++k) {
        const bool odd = (k & 1) != 0;
        const bool epi = b->mean_every > 0 && k == 0;   // chunks start at multiples of mean_every
        switch (b->storage) {
        case LBM_F64: launch_batch_step_f64(b->launch, odd, epi, b->plain, b->own); break;
        case LBM_F32: launch_batch_step_f32(b->launch, odd, epi, b->plain, b->own); break;
        case LBM_F16S: launch_batch_step_f16(b->launch, odd, epi, b->plain, b->own); break;
        case LBM_BF16S: launch_batch_step_bf16(b->launch, odd, epi, b->plain, b->own); break;
        default: launch_batch_step_f16c(b->launch, odd, epi, b->plain, b->own); break;
        }
    }
    const cudaError_t ce = cudaStreamEndCapture(b->own, &graph);
    if (ce != cudaSuccess) return batch_fail(b, LBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return batch_fail(b, LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    b->live = live;
    b->captures++;
    return LBM_OK;
}

// Bring the member contexts' host bookkeeping to batch time t.
static void batch_sync_members(lbm_batch *b)
{
    for (size_t g = 0; g < b->members.size(); ++g) {
        lbm_ctx *c = b->members[g];
        const int64_t tm = std::min(b->t, b->t_end[g]);
        c->t = tm;
        const lbm_params &p = c->p;
        if (p.mean_every > 0) {
            const int64_t hi = std::min(tm, p.mean_end);
            c->msamples = hi > p.mean_start ? (hi - p.mean_start + p.mean_every - 1) / p.mean_every : 0;
        }
        if (p.force_every > 0) {
            c->force_host.clear();
            c->force_rows_dev = (tm + p.force_every - 1) / p.force_every;
        }
    }
}

extern "C" lbm_status lbm_batch_run(lbm_batch *b, int64_t nsteps)
{
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    for (size_t g = 0; g < b->members.size(); ++g)
        if (b->members[g]->unstable && b->t < b->t_end[g])
            return batch_fail(b, LBM_ERR_STATE, "member " + std::to_string(g) + " is unstable; steps refused");
    const int64_t target = b->t + round_chunk(b, nsteps);
    BCK(cudaEventRecord(b->ev_in, b->user));
    BCK(cudaStreamWaitEvent(b->own, b->ev_in, 0));
    for (size_t g = 0; g < b->members.size(); ++g)
        if (b->t < b->t_end[g]) outflow_record(b->members[g], b->members[g]->args(), (b->t & 1) != 0, b->own);
    while (b->t < target) {
        std::vector<int> live;
        int64_t seg_end = target;
        for (size_t g = 0; g < b->members.size(); ++g)
            if (b->t < b->t_end[g]) {
                live.push_back((int)g);
                seg_end = std::min(seg_end, b->t_end[g]);
            }
        if (live.empty()) break;
        if (!b->graph || live != b->live) {
            lbm_status st = batch_rebuild(b, live);
            if (st != LBM_OK) return st;
        }
        const int64_t chunks = (seg_end - b->t) / b->chunk;
        for (int64_t k = 0; k < chunks; ++k) BCK(cudaGraphLaunch(b->graph, b->own));
        int64_t cells = 0;
        for (int g : live) cells += b->members[g]->n_fluid;
        b->updates += cells * (seg_end - b->t);
        b->graph_launches += chunks;
        b->kernel_launches += chunks * b->chunk *
                              (2 + (b->launch.edge_blocks + b->launch.w_blocks > 0 ? 1 : 0) +
                               (b->launch.out_chunks > 0 ? 1 : 0) +
                               (b->launch.q_blocks > 0 ? 1 : 0));
        b->t = seg_end;
    }
    BCK(cudaEventRecord(b->ev_out, b->own));
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0));
    batch_sync_members(b);
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_run_to_end(lbm_batch *b)
{
    if (!b) return LBM_ERR_ARG;
    int64_t te = 0;
    for (int64_t v : b->t_end) te = std::max(te, v);
    if (te >= INT64_MAX / 4) return batch_fail(b, LBM_ERR_STATE, "member ends not set");
    return te > b->t ? lbm_batch_run(b, te - b->t) : LBM_OK;
}

extern "C" lbm_status lbm_batch_sync(lbm_batch *b)
{
    if (!b) return LBM_ERR_ARG;
    BCK(cudaStreamSynchronize(b->own));
    for (size_t g = 0; g < b->members.size(); ++g) {
        const lbm_status st = lbm_sync(b->members[g]);
        if (st != LBM_OK) return batch_fail(b, st, "member " + std::to_string(g) + ": " + b->members[g]->err);
    }
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_get_info(const lbm_batch *b, lbm_batch_info *out)
{
    if (!b || !out) return LBM_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->t = b->t;
    out->chunk = b->chunk;
    out->members = (int32_t)b->members.size();
    for (size_t g = 0; g < b->members.size(); ++g) out->live += b->t < b->t_end[g];
    out->block_x = b->block_x;
    out->block_y = b->block_y;
    out->graph_captures = b->captures;
    out->graph_launches = b->graph_launches;
    out->kernel_launches = b->kernel_launches;
    out->lattice_updates = b->updates;
    return LBM_OK;
}

static lbm_status batch_reset(lbm_batch *b)
{
    BCK(cudaStreamSynchronize(b->own));
    for (lbm_ctx *c : b->members) {
        const lbm_status st = lbm_reset(c);
        if (st != LBM_OK) return st;
    }
    BCK(cudaMemset(b->d_t, 0, sizeof(int64_t)));
    b->t = 0;
    b->updates = 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_batch_autotune(lbm_batch *b, int32_t trials, int32_t *best_bx, int32_t *best_by,
                                         double *best_ms)
{
    if (!b || trials < 1) return LBM_ERR_ARG;
    int64_t cells = 0;
    for (lbm_ctx *c : b->members) cells += c->L.n;
    char what[256];
    std::snprintf(what, sizeof what, "batch|s%d|p%d|n%zu|cells%lld", b->storage, (int)b->plain, b->members.size(),
                  (long long)cells);
    const std::string key = tune_key(what);
    int bx = 0, by = 0;
    double ms = 0;
    if (!tune_lookup(key, &bx, &by, &ms)) {
        std::vector<int64_t> saved = b->t_end;
        std::vector<int64_t> big(b->members.size(), INT64_MAX / 4);
        b->t_end = big;
        cudaEvent_t e0, e1;
        BCK(cudaEventCreate(&e0));
        BCK(cudaEventCreate(&e1));
        double best = 1e300;
        for (int c = 0; c < N_TUNE_CAND; ++c) {
            b->block_x = TUNE_CAND[c][0];
            b->block_y = TUNE_CAND[c][1];
            b->graph_launches = 0;
            lbm_status st = lbm_batch_run(b, b->chunk);          // capture + warm-up
            if (st == LBM_OK) {
                cudaEventRecord(e0, b->user);
                st = lbm_batch_run(b, (int64_t)trials * b->chunk);
                cudaEventRecord(e1, b->user);
            }
            if (st != LBM_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                b->t_end = saved;
                return st != LBM_OK ? st : batch_fail(b, LBM_ERR_CUDA, "autotune timing failed");
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            const double per = t / ((double)trials * b->chunk);
            if (per < best) { best = per; bx = b->block_x; by = b->block_y; }
            if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->t_end = saved;
        ms = best;
        tune_store(key, bx, by, ms);
    }
    b->block_x = bx;
    b->block_y = by;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    b->live.clear();
    b->graph_launches = b->kernel_launches = 0;
    if (best_bx) *best_bx = bx;
    if (best_by) *best_by = by;
    if (best_ms) *best_ms = ms;
    return batch_reset(b);
}

extern "C" const char *lbm_last_error(const lbm_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

extern "C" const char *lbm_status_string(lbm_status s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_UNSTABLE: return "unstable state";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_STATE: return "invalid state for this call";
    case LBM_ERR_IO: return "checkpoint I/O error";
    }
    return "unknown status";
}
