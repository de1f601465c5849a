// lbm_step.cuh -- the fused stream + collide step in the AA pattern.
//
// One array of 27 shifted populations per cell is updated in place:
//   even t: cell x reads slot i of itself, collides, and writes post-collision
//           population i into slot 26-i of itself (purely local);
//   odd  t: cell x gathers population i from slot 26-i of x - c_i, collides,
//           and scatters population i into slot i of x + c_i.
// Boundary links redirect both the gather and the scatter to the cell's own
// slot i (bounce-back and its inlet/outlet variants), so the set of memory
// locations a cell reads is exactly the set it writes and cells never race.
//
// Cells are split in classes: bulk cells (all 26 neighbours are in-domain
// fluid, or the only boundary links cross one x face) take the branch-free
// kernel below with fully coalesced accesses; edge cells (an obstacle, a
// periodic wrap, or both an x face and a wall next to them) go through a
// compact list and the general kernel; wall cells (rows next to a no-slip
// lateral wall) take the bulk access pattern in extra blocks of the edge
// kernel's launch, one block per row segment.
#pragma once

#include "lbm_device.cuh"
#include "sm_count.h"

namespace lbm {

// Per-step outputs of the epilogues (null when not produced this step).
struct StepOut {
    double *msum;           // mean sums [4][n]
    float *snap;            // full-resolution float4 snapshot target
    double *fpart;          // force partials per edge block
    unsigned int *fcount;   // arrival counter of the force reduction
    double *fout;           // force row of this step
};

__device__ __forceinline__ StepOut step_out(const StepArgs &a)
{
    return StepOut{a.msum, a.snap, a.fpart, a.fcount, a.fout};
}

template <class R>
__device__ __forceinline__ void epilogue(const StepArgs &a, const StepOut &o, int64_t c, R drho, R ux, R uy, R uz)
{
    if (o.msum) {
        o.msum[c] += (double)drho;
        o.msum[a.n + c] += (double)ux;
        o.msum[2 * a.n + c] += (double)uy;
        o.msum[3 * a.n + c] += (double)uz;
        if (a.stats) {
            const double x = (double)ux, y = (double)uy, z = (double)uz;
            double *q = o.msum + 4 * a.n + c;
            q[0] += x * x;
            q[a.n] += y * y;
            q[2 * a.n] += z * z;
            q[3 * a.n] += x * y;
            q[4 * a.n] += x * z;
            q[5 * a.n] += y * z;
        }
    }
    if (o.snap) {
        float4 v = make_float4((float)ux, (float)uy, (float)uz, (float)(drho * R(1.0 / 3.0)));
        reinterpret_cast<float4 *>(o.snap)[c] = v;
    }
}

// Bulk cells, one cell per thread, grid (ceil(nx / blockDim.x), ny, nz)
// covering whole rows.  The inlet/outlet cells of a row (x = 0 and x = nx-1
// with class CELL_XFACE) are updated here too, so that their sectors are
// fetched together with the rest of the row: only the first and the last
// warp of a row hold such a lane, and those warps (a warp-uniform condition)
// take the variant of the gather and scatter that redirects the links through
// the x face to the cell's own slot, like the edge kernel; every other warp
// runs the plain gather/scatter.  Contexts created with xface_edge send
// those cells through the boundary records instead (xface_bulk = 0).
template <class S, bool ODD, bool EPI, bool PLAIN>
__device__ __forceinline__ void bulk_cell(const StepArgs &a, const StepOut &o, int x, int y, int z)
{
    using T = Store<S>;
    using R = typename T::R;
    const int64_t c = (int64_t)x + (int64_t)a.nx * ((int64_t)y + (int64_t)a.ny * z);
    const uint8_t fl = a.flags[c];
    if (fl != 0 && fl != CELL_XFACE) return;   // solid or edge cell
    // warp-uniform: does this warp hold x = 0 or x = nx - 1?
    const int xw = x - (int)(threadIdx.x & 31u);
    const bool face_warp = a.xface_bulk && (xw == 0 || xw + 32 > a.nx - 1);
    const bool lo = fl == CELL_XFACE && x == 0;
    const bool hi = fl == CELL_XFACE && x == a.nx - 1;
    const int lo_kind = a.face_x_lo == FACE_INLET ? LINK_INLET : LINK_WALL;
    const int hi_kind = a.face_x_hi == FACE_OUTLET ? LINK_OUTLET : LINK_WALL;
    S *p = static_cast<S *>(a.pdf);
    R *ub = static_cast<R *>(a.ub);
    const int64_t pl = 3 * ((int64_t)y + (int64_t)a.ny * z);
    const char *q = reinterpret_cast<const char *>(p) + c * (int64_t)sizeof(S);
    const int64_t *gof = a.boff[ODD ? 2 : 0], *sof = a.boff[ODD ? 3 : 1];
    R f[Q];
    if (ODD && face_warp) {
        const R ubx = hi ? ub[pl] : R(0), uby = hi ? ub[pl + 1] : R(0), ubz = hi ? ub[pl + 2] : R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            // links through the low face have cx = +1, through the high face cx = -1
            const bool redirect = (cx_of(i) == 1 && lo) || (cx_of(i) == -1 && hi);
            const S *src = redirect ? reinterpret_cast<const S *>(q + a.boff[0][i])
                                    : reinterpret_cast<const S *>(q + gof[i]);
            const R v = T::ld(src);
            f[i] = !redirect ? v : (lo ? boundary_value<R>(a, lo_kind, i, v, R(0), R(0), R(0))
                                       : boundary_value<R>(a, hi_kind, i, v, ubx, uby, ubz));
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = T::ld(reinterpret_cast<const S *>(q + gof[i]));
    }
    R drho, ux, uy, uz;
    collide<R, PLAIN>(f, rates_of<R>(a), drho, ux, uy, uz);
    check_density(drho, a.status);
    // the outlet condition of the next (odd) step uses this step's velocity
    if (!ODD && hi && a.face_x_hi == FACE_OUTLET) {
        ub[pl] = ux;
        ub[pl + 1] = uy;
        ub[pl + 2] = uz;
    }
    if (ODD && face_warp) {
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            // population j leaves through the low face when cx_j = -1, through
            // the high face when cx_j = +1; it returns into i = 26 - j
            const int i = Q - 1 - j;
            const bool redirect = (cx_of(j) == -1 && lo) || (cx_of(j) == 1 && hi);
            S *dst = redirect ? reinterpret_cast<S *>(const_cast<char *>(q) + a.boff[0][i])
                              : reinterpret_cast<S *>(const_cast<char *>(q) + sof[j]);
            const R v = !redirect ? f[j] : (lo ? boundary_value<R>(a, lo_kind, i, f[j], ux, uy, uz)
                                               : boundary_value<R>(a, hi_kind, i, f[j], ux, uy, uz));
            T::st(dst, v);
        }
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) T::st(reinterpret_cast<S *>(const_cast<char *>(q) + sof[j]), f[j]);
    }
    // time average and snapshot after the scatter: the populations are no
    // longer live, which keeps the epilogue variants at the register count of
    // the plain kernel
    if (EPI) epilogue<R>(a, o, c, drho, ux, uy, uz);
}

// Blocks per SM asked of the register allocator (256-thread blocks): the
// 16-bit kernels of the plain collision are bound by instruction issue and
// take 40 registers (six blocks) without the epilogue; FP32 runs its odd
// step at 40 and its even step at 48 (five blocks), the bandwidth each
// measured best at; the general collision 64 (four), FP64 the plain
// collision 80 (three).  Each at no or one spilled value.
template <class S, bool ODD, bool EPI, bool PLAIN>
constexpr int bulk_min_blocks()
{
    return sizeof(S) == 8 ? (PLAIN ? 3 : 1)
                          : (!PLAIN ? 4 : (EPI ? 5 : ((sizeof(S) == 4 && !ODD) ? 5 : 6)));
}

// Single-grid bulk kernel: grid (ceil(nx / blockDim.x), ceil(ny / blockDim.y), nz).
template <class S, bool ODD, bool EPI, bool PLAIN>
__global__ void __launch_bounds__(256, (bulk_min_blocks<S, ODD, EPI, PLAIN>())) k_step_bulk(StepArgs a)
{
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int y = (int)(blockIdx.y * blockDim.y + threadIdx.y);
    if (x >= a.nx || y >= a.ny) return;
    bulk_cell<S, ODD, EPI, PLAIN>(a, step_out(a), x, y, (int)blockIdx.z);
}

// Directions whose component `axis` (0 = x, 1 = y, 2 = z) equals `sign`, as
// a 27-bit mask.
__host__ __device__ constexpr uint32_t dir_mask(int axis, int sign)
{
    uint32_t m = 0;
    for (int i = 0; i < Q; ++i)
        if ((axis == 0 ? cx_of(i) : (axis == 1 ? cy_of(i) : cz_of(i))) == sign) m |= 1u << i;
    return m;
}

// Wall cells (class CELL_WALL): the bulk update with halfway bounce-back on
// the links that cross a lateral wall.  In the odd step such a link gathers
// the cell's own slot i (written by the previous step with the post-collision
// population 26 - i) and the population heading into the wall returns into
// the own slot; the even step is local, as for every cell.  A row's cells
// share y and z, so the wall mask is uniform over a block.  The epilogue
// checks its targets at run time (EPI = true) like the edge kernel's.
template <class S, bool ODD, bool EPI, bool PLAIN>
__device__ __forceinline__ void wall_cell(const StepArgs &a, const StepOut &o, int x, int y, int z)
{
    using T = Store<S>;
    using R = typename T::R;
    const int64_t c = (int64_t)x + (int64_t)a.nx * ((int64_t)y + (int64_t)a.ny * z);
    if (a.flags[c] != CELL_WALL) return;
    const char *q = reinterpret_cast<const char *>(a.pdf) + c * (int64_t)sizeof(S);
    const int64_t *gof = a.boff[ODD ? 2 : 0], *sof = a.boff[ODD ? 3 : 1];
    // bit i: the link of pull direction i (from x - c_i) crosses a wall
    const uint32_t wmask = (y == 0 ? dir_mask(1, 1) : 0u) | (y == a.ny - 1 ? dir_mask(1, -1) : 0u) |
                           (z == 0 ? dir_mask(2, 1) : 0u) | (z == a.nz - 1 ? dir_mask(2, -1) : 0u);
    R f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int64_t off = (ODD && ((wmask >> i) & 1u)) ? a.boff[0][i] : gof[i];
        f[i] = T::ld(reinterpret_cast<const S *>(q + off));
    }
    R drho, ux, uy, uz;
    collide<R, PLAIN>(f, rates_of<R>(a), drho, ux, uy, uz);
    check_density(drho, a.status);
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        // population j heads to x + c_j = x - c_i, i = 26 - j
        const int i = Q - 1 - j;
        const int64_t off = (ODD && ((wmask >> i) & 1u)) ? a.boff[0][i] : sof[j];
        T::st(reinterpret_cast<S *>(const_cast<char *>(q) + off), f[j]);
    }
    if (EPI) epilogue<R>(a, o, c, drho, ux, uy, uz);
}

// Sum a double over the block into partials[blockIdx]; the last block to
// arrive adds the partials in a fixed order and writes the result, so the
// value does not depend on block scheduling.
__device__ __forceinline__ void block_force_reduce(const StepOut &o, int64_t blk, int64_t nblk, double fx, double fy,
                                                   double fz, bool add = false)
{
    __shared__ double sh[3][EDGE_BLOCK / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += __shfl_down_sync(0xffffffffu, fx, o);
        fy += __shfl_down_sync(0xffffffffu, fy, o);
        fz += __shfl_down_sync(0xffffffffu, fz, o);
    }
    if (lane == 0) { sh[0][warp] = fx; sh[1][warp] = fy; sh[2][warp] = fz; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[3] = {0, 0, 0};
        for (int w = 0; w < EDGE_BLOCK / 32; ++w)
            for (int d = 0; d < 3; ++d) s[d] += sh[d][w];
        for (int d = 0; d < 3; ++d) o.fpart[3 * blk + d] = s[d];
        __threadfence();
        const unsigned prev = atomicAdd(o.fcount, 1u);
        last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // fixed-order tree: each thread sums a strided subset, then a shared tree
    __shared__ double tr[3][EDGE_BLOCK];
    double s[3] = {0, 0, 0};
    for (int64_t b = threadIdx.x; b < nblk; b += EDGE_BLOCK)
        for (int d = 0; d < 3; ++d) s[d] += ((volatile double *)o.fpart)[3 * b + d];
    for (int d = 0; d < 3; ++d) tr[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int h = EDGE_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int d = 0; d < 3; ++d) tr[d][threadIdx.x] += tr[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) o.fout[d] = add ? o.fout[d] + tr[d][0] : tr[d][0];
        *o.fcount = 0u;
    }
}

// Link code of direction i in an edge record (3 bits per direction, nine
// directions per 32-bit word).
__device__ __forceinline__ int link_code(const uint4 &e, int i)
{
    const uint32_t w = i < 9 ? e.y : (i < 18 ? e.z : e.w);
    return (int)((w >> (3 * (i % 9))) & 7u);
}

// Fluid neighbour x - c_i of cell c reached through a periodic face.
__device__ __forceinline__ int64_t wrapped_neighbour(const StepArgs &a, uint32_t c, int i)
{
    const uint32_t nx = (uint32_t)a.nx, ny = (uint32_t)a.ny;
    const uint32_t yz = c / nx;
    int x = (int)(c - yz * nx), y = (int)(yz % ny), z = (int)(yz / ny);
    x -= cx_of(i); y -= cy_of(i); z -= cz_of(i);
    x = x < 0 ? x + a.nx : (x >= a.nx ? x - a.nx : x);
    y = y < 0 ? y + a.ny : (y >= a.ny ? y - a.ny : y);
    z = z < 0 ? z + a.nz : (z >= a.nz ? z - a.nz : z);
    return (int64_t)x + (int64_t)a.nx * ((int64_t)y + (int64_t)a.ny * z);
}

// Edge cells: one thread per record of the compact list; the link codes were
// classified once at creation.
template <class S, bool ODD, bool PLAIN>
__device__ __forceinline__ void edge_cell(const StepArgs &a, const StepOut &o, int64_t k,
                                          typename Store<S>::R &fx, typename Store<S>::R &fy,
                                          typename Store<S>::R &fz)
{
    using T = Store<S>;
    using R = typename T::R;
    {
        const uint4 e = a.edge[k];
        const uint32_t c32 = e.x;
        const int64_t c = c32;
        const uint32_t yz = c32 / (uint32_t)a.nx;          // y + ny * z
        const int x = (int)(c32 - yz * (uint32_t)a.nx);
        S *p = static_cast<S *>(a.pdf);
        R *ub = static_cast<R *>(a.ub);
        const int64_t pl = 3 * (int64_t)yz;
        R f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (ODD) {
                const int kind = link_code(e, i);
                if (kind == LINK_FLUID || kind == LINK_WRAP) {
                    const int64_t off = cx_of(i) + (int64_t)cy_of(i) * a.nx + (int64_t)cz_of(i) * a.nxy;
                    const int64_t nbr = kind == LINK_FLUID ? c - off : wrapped_neighbour(a, c32, i);
                    f[i] = T::ld(p + (int64_t)(Q - 1 - i) * a.slot + nbr);
                } else {
                    const R own = T::ld(p + (int64_t)i * a.slot + c);
                    f[i] = (kind == LINK_OUTLET) ? boundary_value<R>(a, kind, i, own, ub[pl], ub[pl + 1], ub[pl + 2])
                                                 : boundary_value<R>(a, kind, i, own, R(0), R(0), R(0));
                }
            } else {
                f[i] = T::ld(p + (int64_t)i * a.slot + c);
            }
        }
        R drho, ux, uy, uz;
        collide<R, PLAIN>(f, rates_of<R>(a), drho, ux, uy, uz);
        check_density(drho, a.status);
        epilogue<R>(a, o, c, drho, ux, uy, uz);
        // the outlet condition of the next (odd) step uses this step's velocity
        if (!ODD && x == a.nx - 1 && a.face_x_hi == FACE_OUTLET) {
            ub[pl] = ux;
            ub[pl + 1] = uy;
            ub[pl + 2] = uz;
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            // population j heads to x + c_j = x - c_i with i = 26 - j
            const int i = Q - 1 - j;
            const int kind = link_code(e, i);
            if (kind == LINK_SOLID) {   // momentum exchange with the obstacle
                if (cx_of(j)) fx += R(2 * cx_of(j)) * f[j];
                if (cy_of(j)) fy += R(2 * cy_of(j)) * f[j];
                if (cz_of(j)) fz += R(2 * cz_of(j)) * f[j];
            }
            if (ODD) {
                if (kind == LINK_FLUID || kind == LINK_WRAP) {
                    const int64_t off = cx_of(j) + (int64_t)cy_of(j) * a.nx + (int64_t)cz_of(j) * a.nxy;
                    const int64_t nbr = kind == LINK_FLUID ? c + off : wrapped_neighbour(a, c32, i);
                    T::st(p + (int64_t)j * a.slot + nbr, f[j]);
                } else {
                    // returns through the boundary into direction i of this cell
                    const R v = boundary_value<R>(a, kind, i, f[j], ux, uy, uz);
                    T::st(p + (int64_t)i * a.slot + c, v);
                }
            } else {
                T::st(p + (int64_t)(Q - 1 - j) * a.slot + c, f[j]);
            }
        }
    }
}

static_assert(WALL_BLOCK == EDGE_BLOCK, "wall-row blocks run in the edge kernel's launch");

// Single-grid edge kernel: blocks [0, eblocks) take one record of the compact
// list per thread; the blocks after them take the wall rows, block b covering
// cells [(b % wx) WALL_BLOCK, ...) of wall row b / wx (they have no obstacle
// links and stay out of the force reduction).
template <class S, bool ODD, bool PLAIN>
__global__ void __launch_bounds__(EDGE_BLOCK) k_step_edge(StepArgs a, int eblocks, int wx)
{
    using R = typename Store<S>::R;
    const StepOut o = step_out(a);
    if ((int)blockIdx.x >= eblocks) {
        const int64_t b = (int64_t)blockIdx.x - eblocks, r = b / wx;
        const int x = (int)(b - r * wx) * WALL_BLOCK + (int)threadIdx.x;
        if (x < a.nx) {
            int y, z;
            wall_row_yz(r, a.ny, a.nz, y, z);
            wall_cell<S, ODD, true, PLAIN>(a, o, x, y, z);
        }
        return;
    }
    const int64_t k = (int64_t)blockIdx.x * EDGE_BLOCK + threadIdx.x;
    R fx = R(0), fy = R(0), fz = R(0);     // this cell's obstacle force
    if (k < a.n_edge) edge_cell<S, ODD, PLAIN>(a, o, k, fx, fy, fz);
    if (o.fpart) block_force_reduce(o, blockIdx.x, eblocks, (double)fx, (double)fy, (double)fz);
}

// Convective outflow, between steps (one thread per outlet column y, z).
// fix: each fluid outlet cell x_b gets, for its links through the x-high face
// (cx = -1, the source not beyond a lateral wall),
//     f_i = c_s f_i(x_b - e_x) + (1 - c_s) f_i(x_b)
// from the pre-collision populations of the step just taken (recorded by the
// previous call), written into its own slot i: where the next step, of
// either parity, reads that link.  A solid (or missing) inner neighbour makes
// the cell extrapolate from itself.
// record: the populations with cx = -1 that the next step (parity next_odd)
// will gather, of the outlet cell (all such links of an outlet cell are
// boundary links: its own slot) and of the cell next to it (own slot for an
// even step or a boundary link; slot 26 - i of the source for an odd step).
// The fix only writes outlet-cell slots of cx = -1, which the inner cell's
// gather never reads.
template <class S>
__device__ __forceinline__ void outflow_link(const StepArgs &a, int64_t yz, int k, bool fix, bool next_odd)
{
    using T = Store<S>;
    using R = typename T::R;
    const int64_t P = (int64_t)a.ny * a.nz;
    const int64_t c = (int64_t)(a.nx - 1) + (int64_t)a.nx * yz;
    if (a.flags[c] & CELL_SOLID) return;
    const int y = (int)(yz % a.ny), z = (int)(yz / a.ny);
    const int i = 3 * k;                                    // cx = -1
    R *own = static_cast<R *>(a.ob) + (int64_t)k * P + yz;
    R *in = own + 9 * P;
    const bool inner = a.nx >= 2 && !(a.flags[c - 1] & CELL_SOLID);
    S *p = static_cast<S *>(a.pdf);
    int sy = y - cy_of(i), sz = z - cz_of(i);
    bool through_face = true;                              // the link leaves through the x face, not a wall
    if (sy < 0 || sy >= a.ny) { through_face = a.face_y == FACE_PERIODIC; sy = sy < 0 ? sy + a.ny : sy - a.ny; }
    if (sz < 0 || sz >= a.nz) { through_face = through_face && a.face_z == FACE_PERIODIC; sz = sz < 0 ? sz + a.nz : sz - a.nz; }
    R mine;
    if (fix && through_face) {
        const R cs = R(0.57735026918962576451);
        mine = cs * (inner ? *in : *own) + (R(1) - cs) * *own;
        T::st(p + (int64_t)i * a.slot + c, mine);
        mine = T::ld(p + (int64_t)i * a.slot + c);         // the stored (rounded) value
    } else {
        mine = T::ld(p + (int64_t)i * a.slot + c);
    }
    *own = mine;                                            // every cx = -1 link of an outlet cell reads its own slot
    if (!inner) return;
    int64_t src = -1;
    if (next_odd && through_face) {                         // the inner cell's source (nx - 1, y - cy, z - cz)
        const int64_t s2 = (int64_t)(a.nx - 1) + (int64_t)a.nx * ((int64_t)sy + (int64_t)a.ny * sz);
        if (!(a.flags[s2] & CELL_SOLID)) src = s2;
    }
    *in = src >= 0 ? T::ld(p + (int64_t)(Q - 1 - i) * a.slot + src) : T::ld(p + (int64_t)i * a.slot + c - 1);
}

// One thread per outlet column and direction (nine per column: the plane is
// strided by nx in memory, so many accesses must be in flight).
template <class S>
__global__ void __launch_bounds__(256) k_outflow(StepArgs a, int fix, int next_odd)
{
    const int64_t P = (int64_t)a.ny * a.nz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 9 * P; t += (int64_t)gridDim.x * blockDim.x)
        outflow_link<S>(a, t % P, (int)(t / P), fix != 0, next_odd != 0);
}

template <class S>
static void launch_outflow(const StepArgs &a, bool fix, bool next_odd, cudaStream_t s)
{
    if (a.face_x_hi != FACE_OUTFLOW) return;
    const int64_t P = (int64_t)a.ny * a.nz;
    k_outflow<S><<<(unsigned)std::min<int64_t>((9 * P + 255) / 256, gb300::sm_count() * 16), 256, 0, s>>>(a, fix ? 1 : 0,
                                                                                          next_odd ? 1 : 0);
}

// Interpolated bounce-back (Bouzidi, Firdaouss & Lallemand 2001), after the
// step: for an obstacle link of fluid cell x (pull direction i, j = 26 - i
// heading into the wall at fraction q of the link, x1 = x + c_i and
// x2 = x + 2 c_i behind it) the own slot i holds f*_j(x), the halfway
// bounce-back value, and f*_j(x1), f*_j(x2), f*_i(x), f*_i(x1) sit where
// the next step gathers them: for a next odd step slot i of x1 / x2 and slot
// j of x / x1, for a next even step slot j of x / x1 and slot i of x1 / x2.
// None of those slots belongs to an obstacle link, so the links are updated
// in place without ordering.  The returned population replaces own slot i;
// the momentum exchange gains c_j (f_returned - f*_j) over the halfway value
// recorded by the edge kernel.
template <class S>
__device__ __forceinline__ void qbb_link(const StepArgs &a, int64_t k, bool next_odd, typename Store<S>::R &fx,
                                         typename Store<S>::R &fy, typename Store<S>::R &fz)
{
    using T = Store<S>;
    using R = typename T::R;
    S *p = static_cast<S *>(a.pdf);
    const uint4 e = a.qlinks[k];
    const int i = (int)(e.w & 0xFFu), mode = (int)(e.w >> 8), j = Q - 1 - i;
    const int64_t x = e.x, x1 = e.y, x2 = e.z;
    const int64_t si = (int64_t)i * a.slot, sj = (int64_t)j * a.slot;
    const R q = R(a.qval[k]);
    const R a0 = T::ld(p + si + x);
    R ret;
    if (q < R(0.5)) {
        const R a1 = T::ld(p + (next_odd ? si + x1 : sj + x));
        if (mode == 2) {
            const R a2 = T::ld(p + (next_odd ? si + x2 : sj + x1));
            ret = q * (R(1) + R(2) * q) * a0 + (R(1) - R(4) * q * q) * a1 - q * (R(1) - R(2) * q) * a2;
        } else {
            ret = R(2) * q * a0 + (R(1) - R(2) * q) * a1;
        }
    } else {
        const R b0 = T::ld(p + (next_odd ? sj + x : si + x1));
        if (mode == 2) {
            const R b1 = T::ld(p + (next_odd ? sj + x1 : si + x2));
            ret = a0 / (q * (R(2) * q + R(1))) + (R(2) * q - R(1)) / q * b0 -
                  (R(2) * q - R(1)) / (R(2) * q + R(1)) * b1;
        } else {
            ret = a0 / (R(2) * q) + (R(2) * q - R(1)) / (R(2) * q) * b0;
        }
    }
    T::st(p + si + x, ret);
    const R dv = ret - a0;
    fx += R(cx_of(j)) * dv;
    fy += R(cy_of(j)) * dv;
    fz += R(cz_of(j)) * dv;
}

template <class S>
__global__ void __launch_bounds__(EDGE_BLOCK) k_qbb(StepArgs a, int next_odd)
{
    using R = typename Store<S>::R;
    const int64_t k = (int64_t)blockIdx.x * EDGE_BLOCK + threadIdx.x;
    R fx = R(0), fy = R(0), fz = R(0);
    if (k < a.n_qlinks) qbb_link<S>(a, k, next_odd != 0, fx, fy, fz);
    if (a.fout) {
        StepOut o{nullptr, nullptr, a.qpart, a.qcount, a.fout};
        block_force_reduce(o, blockIdx.x, gridDim.x, (double)fx, (double)fy, (double)fz, true);
    }
}

template <class S>
static void launch_qbb(const StepArgs &a, bool next_odd, cudaStream_t s)
{
    if (a.n_qlinks <= 0) return;
    k_qbb<S><<<(unsigned)((a.n_qlinks + EDGE_BLOCK - 1) / EDGE_BLOCK), EDGE_BLOCK, 0, s>>>(a, next_odd ? 1 : 0);
}

template <class S, bool ODD, bool EPI, bool PLAIN>
static void launch_bulk(const StepArgs &a, int block_x, int block_y, cudaStream_t s, cudaEvent_t ev_interior)
{
    const dim3 grd((a.nx + block_x - 1) / block_x, (a.ny + block_y - 1) / block_y, a.nz);
    k_step_bulk<S, ODD, EPI, PLAIN><<<grd, dim3(block_x, block_y), 0, s>>>(a);
    if (ev_interior) cudaEventRecord(ev_interior, s);
}

// ---------------------------------------------------------------------------
// batched launches: one bulk and one edge launch per step over every member
// lattice of a batch.  Blocks are numbered member after member; a block finds
// its member by binary search over the members' first block numbers.
// Quantities that depend on the step (time-average sampling, force row) come
// from the device step counter, so a captured sequence of steps can be
// replayed unchanged.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_member(const int64_t *begin, int nm, int64_t b)
{
    int lo = 0, hi = nm - 1;                 // largest m with begin[m] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool samples_at(const BatchMember &B, int64_t t)
{
    return B.msum && B.mean_every > 0 && t >= B.mean_start && t < B.mean_end && (t - B.mean_start) % B.mean_every == 0;
}

template <class S, bool ODD, bool EPI, bool PLAIN>
__global__ void __launch_bounds__(256, (bulk_min_blocks<S, ODD, EPI, PLAIN>())) k_batch_bulk(const BatchMember *mem, const int64_t *begin, int nm,
                                                    const int64_t *tdev)
{
    // the member's step arguments are staged in shared memory: the cell
    // update reads its 54 access offsets from there (a broadcast per access)
    // rather than from the global member table
    __shared__ StepArgs sa;
    const int m = find_member(begin, nm, blockIdx.x);
    const BatchMember &B = mem[m];
    {
        static_assert(sizeof(StepArgs) % 8 == 0, "StepArgs is copied as 8-byte words");
        const int tid = (int)(threadIdx.x + threadIdx.y * blockDim.x), nt = (int)(blockDim.x * blockDim.y);
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&B.a);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sa);
        for (int k = tid; k < (int)(sizeof(StepArgs) / 8); k += nt) dst[k] = src[k];
    }
    __syncthreads();
    const int64_t local = (int64_t)blockIdx.x - begin[m];
    const int bx = (int)(local % B.gx);
    const int64_t r = local / B.gx;
    const int by = (int)(r % B.gy);
    const int z = (int)(r / B.gy);
    const int x = bx * (int)blockDim.x + (int)threadIdx.x;
    const int y = by * (int)blockDim.y + (int)threadIdx.y;
    if (x >= sa.nx || y >= sa.ny) return;
    StepOut o{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (EPI && samples_at(B, *tdev)) o.msum = B.msum;
    bulk_cell<S, ODD, EPI, PLAIN>(sa, o, x, y, z);
}

// Batched edge kernel: blocks [0, eblocks) are the members' edge blocks,
// the blocks after them the members' wall-row blocks (numbered by w_begin).
template <class S, bool ODD, bool PLAIN>
__global__ void __launch_bounds__(EDGE_BLOCK) k_batch_edge(const BatchMember *mem, const int64_t *begin, int nm,
                                                           const int64_t *tdev, int epi, int64_t eblocks,
                                                           const int64_t *w_begin)
{
    using R = typename Store<S>::R;
    if ((int64_t)blockIdx.x >= eblocks) {
        const int64_t b = (int64_t)blockIdx.x - eblocks;
        const int m = find_member(w_begin, nm, b);
        const BatchMember &B = mem[m];
        const int64_t local = b - w_begin[m], r = local / B.wx;
        const int x = (int)(local - r * B.wx) * WALL_BLOCK + (int)threadIdx.x;
        if (x >= B.a.nx) return;
        int y, z;
        wall_row_yz(r, B.a.ny, B.a.nz, y, z);
        StepOut o{nullptr, nullptr, nullptr, nullptr, nullptr};
        if (epi && samples_at(B, *tdev)) o.msum = B.msum;
        wall_cell<S, ODD, true, PLAIN>(B.a, o, x, y, z);
        return;
    }
    const int m = find_member(begin, nm, blockIdx.x);
    const BatchMember &B = mem[m];
    const int64_t lb = (int64_t)blockIdx.x - begin[m], nb = begin[m + 1] - begin[m];
    const int64_t k = lb * EDGE_BLOCK + threadIdx.x;
    const int64_t t = *tdev;
    StepOut o{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (epi && samples_at(B, t)) o.msum = B.msum;
    if (B.force && t % B.force_every == 0) {
        o.fpart = B.a.fpart;
        o.fcount = B.a.fcount;
        o.fout = B.force + 3 * (t / B.force_every);
    }
    R fx = R(0), fy = R(0), fz = R(0);
    if (k < B.a.n_edge) edge_cell<S, ODD, PLAIN>(B.a, o, k, fx, fy, fz);
    if (o.fpart) block_force_reduce(o, lb, nb, (double)fx, (double)fy, (double)fz);
}

// End of a batched step: the convective outflow of every member with that
// outlet (grid x = member, grid y splits its outlet plane) ...
template <class S>
__global__ void __launch_bounds__(256) k_batch_outflow(const BatchMember *mem, int nm, int fix, int next_odd)
{
    const StepArgs &a = mem[blockIdx.x].a;
    if (a.face_x_hi != FACE_OUTFLOW) return;
    const int64_t P = (int64_t)a.ny * a.nz;
    for (int64_t t = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; t < 9 * P; t += (int64_t)gridDim.y * blockDim.x)
        outflow_link<S>(a, t % P, (int)(t / P), fix != 0, next_odd != 0);
}

// ... then the interpolated bounce-back of the members with wall distances
// (blocks numbered member after member, as for the edge kernel), each
// member's force correction reduced over its blocks in a fixed order and
// added to its force row of this step.
template <class S>
__global__ void __launch_bounds__(EDGE_BLOCK) k_batch_qbb(const BatchMember *mem, const int64_t *begin, int nm,
                                                         const int64_t *tdev, int next_odd)
{
    using R = typename Store<S>::R;
    const int m = find_member(begin, nm, blockIdx.x);
    const BatchMember &B = mem[m];
    const int64_t lb = (int64_t)blockIdx.x - begin[m], nb = begin[m + 1] - begin[m];
    const int64_t k = lb * EDGE_BLOCK + threadIdx.x;
    R fx = R(0), fy = R(0), fz = R(0);
    if (k < B.a.n_qlinks) qbb_link<S>(B.a, k, next_odd != 0, fx, fy, fz);
    const int64_t t = *tdev;
    if (B.force && t % B.force_every == 0) {
        StepOut o{nullptr, nullptr, B.a.qpart, B.a.qcount, B.force + 3 * (t / B.force_every)};
        block_force_reduce(o, lb, nb, (double)fx, (double)fy, (double)fz, true);
    }
}

static __global__ void k_batch_tick(int64_t *t)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t += 1;
}

template <class S>
void launch_batch_step_t(const BatchLaunch &L, bool odd, bool epi, bool plain, cudaStream_t s)
{
    const dim3 blk(L.block_x, L.block_y);
    const unsigned nb = (unsigned)L.bulk_blocks, ne = (unsigned)(L.edge_blocks + L.w_blocks);
#define LBM_BB(O, E, P) k_batch_bulk<S, O, E, P><<<nb, blk, 0, s>>>(L.mem, L.bulk_begin, L.nm, L.t)
    if (plain) {
        if (odd) { if (epi) LBM_BB(true, true, true); else LBM_BB(true, false, true); }
        else     { if (epi) LBM_BB(false, true, true); else LBM_BB(false, false, true); }
    } else {
        if (odd) { if (epi) LBM_BB(true, true, false); else LBM_BB(true, false, false); }
        else     { if (epi) LBM_BB(false, true, false); else LBM_BB(false, false, false); }
    }
#undef LBM_BB
    if (ne > 0) {
        if (plain) {
#define LBM_BE(O, P) k_batch_edge<S, O, P><<<ne, EDGE_BLOCK, 0, s>>>(L.mem, L.edge_begin, L.nm, L.t, epi, \
                                                                    L.edge_blocks, L.w_begin)
            if (odd) LBM_BE(true, true); else LBM_BE(false, true);
        } else {
            if (odd) LBM_BE(true, false); else LBM_BE(false, false);
#undef LBM_BE
        }
    }
    if (L.q_blocks > 0)
        k_batch_qbb<S><<<(unsigned)L.q_blocks, EDGE_BLOCK, 0, s>>>(L.mem, L.q_begin, L.nm, L.t, odd ? 0 : 1);
    if (L.out_chunks > 0)
        k_batch_outflow<S><<<dim3((unsigned)L.nm, (unsigned)L.out_chunks), 256, 0, s>>>(L.mem, L.nm, 1, odd ? 0 : 1);
    k_batch_tick<<<1, 32, 0, s>>>(L.t);
}

template <class S>
void launch_step_t(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, int block_y, cudaStream_t s,
                   cudaEvent_t ev_interior, cudaEvent_t ev_bulk)
{
    const cudaEvent_t e = ev_interior;
    const int bx = block_x, by = block_y;
    if (plain) {
        if (odd) { if (epi) launch_bulk<S, true, true, true>(a, bx, by, s, e); else launch_bulk<S, true, false, true>(a, bx, by, s, e); }
        else     { if (epi) launch_bulk<S, false, true, true>(a, bx, by, s, e); else launch_bulk<S, false, false, true>(a, bx, by, s, e); }
    } else {
        if (odd) { if (epi) launch_bulk<S, true, true, false>(a, bx, by, s, e); else launch_bulk<S, true, false, false>(a, bx, by, s, e); }
        else     { if (epi) launch_bulk<S, false, true, false>(a, bx, by, s, e); else launch_bulk<S, false, false, false>(a, bx, by, s, e); }
    }
    if (ev_bulk) cudaEventRecord(ev_bulk, s);
    if (a.n_edge > 0 || a.n_wall > 0) {
        const int eb = (int)((a.n_edge + EDGE_BLOCK - 1) / EDGE_BLOCK);
        const int wx = (a.nx + WALL_BLOCK - 1) / WALL_BLOCK;
        const int64_t wb = a.n_wall > 0 ? (int64_t)wx * wall_rows(a.ny, a.nz) : 0;
        const dim3 eg((unsigned)(eb + wb));
        if (plain) {
            if (odd) k_step_edge<S, true, true><<<eg, EDGE_BLOCK, 0, s>>>(a, eb, wx);
            else     k_step_edge<S, false, true><<<eg, EDGE_BLOCK, 0, s>>>(a, eb, wx);
        } else {
            if (odd) k_step_edge<S, true, false><<<eg, EDGE_BLOCK, 0, s>>>(a, eb, wx);
            else     k_step_edge<S, false, false><<<eg, EDGE_BLOCK, 0, s>>>(a, eb, wx);
        }
    }
    launch_qbb<S>(a, !odd, s);
    launch_outflow<S>(a, true, !odd, s);
}

// Record-only outflow pass for the state before a step of parity `odd`.
template <class S>
void launch_outflow_record_t(const StepArgs &a, bool odd, cudaStream_t s)
{
    launch_outflow<S>(a, false, odd, s);
}

}  // namespace lbm
