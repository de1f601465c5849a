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
// Cells are split in two classes: bulk cells (all 26 neighbours are in-domain
// fluid) take the branch-free kernel below with fully coalesced accesses;
// edge cells (a wall, the inlet/outlet plane, an obstacle or a periodic wrap
// next to them) go through a compact list and the general kernel.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <class R>
__device__ __forceinline__ void epilogue(const StepArgs &a, int64_t c, R drho, R ux, R uy, R uz)
{
    if (a.msum) {
        a.msum[c] += (double)drho;
        a.msum[a.n + c] += (double)ux;
        a.msum[2 * a.n + c] += (double)uy;
        a.msum[3 * a.n + c] += (double)uz;
    }
    if (a.snap) {
        float4 v = make_float4((float)ux, (float)uy, (float)uz, (float)(drho * R(1.0 / 3.0)));
        reinterpret_cast<float4 *>(a.snap)[c] = v;
    }
}

// Bulk cells, one cell per thread, grid (ceil(nx / blockDim.x), ny, nz)
// covering whole rows.  The inlet/outlet cells of a row (x = 0 and x = nx-1
// with class CELL_XFACE) are updated here too, so that their sectors are
// fetched together with the rest of the row: only the first and the last
// warp of a row hold such a lane, and those warps (a warp-uniform condition)
// take the variant of the gather and scatter that redirects the links through
// the x face to the cell's own slot, like the edge kernel; every other warp
// runs the plain gather/scatter.
template <class S, bool ODD, bool EPI, bool PLAIN>
__global__ void __launch_bounds__(256) k_step_bulk(StepArgs a)
{
    using T = Store<S>;
    using R = typename T::R;
    const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= a.nx) return;
    const int y = (int)blockIdx.y;
    const int64_t c = (int64_t)x + (int64_t)a.nx * ((int64_t)y + (int64_t)a.ny * blockIdx.z);
    const uint8_t fl = a.flags[c];
    if (fl != 0 && fl != CELL_XFACE) return;   // solid or edge cell
    // warp-uniform: does this warp hold x = 0 or x = nx - 1?
    const int xw = x - (int)(threadIdx.x & 31u);
    const bool face_warp = xw == 0 || xw + 32 > a.nx - 1;
    const bool lo = fl == CELL_XFACE && x == 0;
    const bool hi = fl == CELL_XFACE && x == a.nx - 1;
    const int lo_kind = a.face_x_lo == FACE_INLET ? LINK_INLET : LINK_WALL;
    const int hi_kind = a.face_x_hi == FACE_OUTLET ? LINK_OUTLET : LINK_WALL;
    S *p = static_cast<S *>(a.pdf);
    R *ub = static_cast<R *>(a.ub);
    const int64_t pl = 3 * ((int64_t)y + (int64_t)a.ny * blockIdx.z);
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
    if (EPI) epilogue<R>(a, c, drho, ux, uy, uz);
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
}

// Sum a double over the block into partials[blockIdx]; the last block to
// arrive adds the partials in a fixed order and writes the result, so the
// value does not depend on block scheduling.
__device__ __forceinline__ void block_force_reduce(const StepArgs &a, double fx, double fy, double fz)
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
        for (int d = 0; d < 3; ++d) a.fpart[3 * (int64_t)blockIdx.x + d] = s[d];
        __threadfence();
        const unsigned prev = atomicAdd(a.fcount, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // fixed-order tree: each thread sums a strided subset, then a shared tree
    __shared__ double tr[3][EDGE_BLOCK];
    double s[3] = {0, 0, 0};
    for (int64_t b = threadIdx.x; b < gridDim.x; b += EDGE_BLOCK)
        for (int d = 0; d < 3; ++d) s[d] += ((volatile double *)a.fpart)[3 * b + d];
    for (int d = 0; d < 3; ++d) tr[d][threadIdx.x] = s[d];
    __syncthreads();
    for (int h = EDGE_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int d = 0; d < 3; ++d) tr[d][threadIdx.x] += tr[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) a.fout[d] = tr[d][0];
        *a.fcount = 0u;
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
__global__ void __launch_bounds__(EDGE_BLOCK) k_step_edge(StepArgs a)
{
    using T = Store<S>;
    using R = typename T::R;
    const int64_t k = (int64_t)blockIdx.x * EDGE_BLOCK + threadIdx.x;
    R fx = R(0), fy = R(0), fz = R(0);     // this cell's obstacle force
    if (k < a.n_edge) {
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
        epilogue<R>(a, c, drho, ux, uy, uz);
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
    if (a.fpart) block_force_reduce(a, (double)fx, (double)fy, (double)fz);
}

template <class S, bool ODD, bool EPI, bool PLAIN>
static void launch_bulk(const StepArgs &a, int block_x, cudaStream_t s, cudaEvent_t ev_interior)
{
    const dim3 grd((a.nx + block_x - 1) / block_x, a.ny, a.nz);
    k_step_bulk<S, ODD, EPI, PLAIN><<<grd, block_x, 0, s>>>(a);
    if (ev_interior) cudaEventRecord(ev_interior, s);
}

template <class S>
void launch_step_t(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, cudaStream_t s,
                   cudaEvent_t ev_interior, cudaEvent_t ev_bulk)
{
    const cudaEvent_t e = ev_interior;
    if (plain) {
        if (odd) { if (epi) launch_bulk<S, true, true, true>(a, block_x, s, e); else launch_bulk<S, true, false, true>(a, block_x, s, e); }
        else     { if (epi) launch_bulk<S, false, true, true>(a, block_x, s, e); else launch_bulk<S, false, false, true>(a, block_x, s, e); }
    } else {
        if (odd) { if (epi) launch_bulk<S, true, true, false>(a, block_x, s, e); else launch_bulk<S, true, false, false>(a, block_x, s, e); }
        else     { if (epi) launch_bulk<S, false, true, false>(a, block_x, s, e); else launch_bulk<S, false, false, false>(a, block_x, s, e); }
    }
    if (ev_bulk) cudaEventRecord(ev_bulk, s);
    if (a.n_edge > 0) {
        const dim3 eg((unsigned)((a.n_edge + EDGE_BLOCK - 1) / EDGE_BLOCK));
        if (plain) {
            if (odd) k_step_edge<S, true, true><<<eg, EDGE_BLOCK, 0, s>>>(a);
            else     k_step_edge<S, false, true><<<eg, EDGE_BLOCK, 0, s>>>(a);
        } else {
            if (odd) k_step_edge<S, true, false><<<eg, EDGE_BLOCK, 0, s>>>(a);
            else     k_step_edge<S, false, false><<<eg, EDGE_BLOCK, 0, s>>>(a);
        }
    }
}

}  // namespace lbm
