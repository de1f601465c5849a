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

// Bulk cells: grid (ceil(nx / blockDim.x), ny, nz), one cell per thread.
template <class S, bool ODD, bool EPI, bool PLAIN>
__global__ void __launch_bounds__(256) k_step_bulk(StepArgs a)
{
    using T = Store<S>;
    using R = typename T::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.nx) return;
    const int64_t c = (int64_t)x + (int64_t)a.nx * ((int64_t)blockIdx.y + (int64_t)a.ny * blockIdx.z);
    if (a.flags[c] != 0) return;   // solid or edge cell
    S *p = static_cast<S *>(a.pdf);
    R f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (ODD) {
            const int64_t off = cx_of(i) + (int64_t)cy_of(i) * a.nx + (int64_t)cz_of(i) * a.nxy;
            f[i] = T::ld(p + (int64_t)(Q - 1 - i) * a.slot + c - off);
        } else {
            f[i] = T::ld(p + (int64_t)i * a.slot + c);
        }
    }
    R drho, ux, uy, uz;
    const Rates rt{a.w1, a.w2, a.w3, a.galilean};
    collide<R, PLAIN>(f, rt, drho, ux, uy, uz);
    check_density(drho, a.status);
    if (EPI) epilogue<R>(a, c, drho, ux, uy, uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (ODD) {
            const int64_t off = cx_of(i) + (int64_t)cy_of(i) * a.nx + (int64_t)cz_of(i) * a.nxy;
            T::st(p + (int64_t)i * a.slot + c + off, f[i]);
        } else {
            T::st(p + (int64_t)(Q - 1 - i) * a.slot + c, f[i]);
        }
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

// Edge cells: one thread per entry of the compact list.
template <class S, bool ODD, bool PLAIN>
__global__ void __launch_bounds__(EDGE_BLOCK) k_step_edge(StepArgs a)
{
    using T = Store<S>;
    using R = typename T::R;
    const int64_t k = (int64_t)blockIdx.x * EDGE_BLOCK + threadIdx.x;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    if (k < a.n_edge) {
        const int64_t c = a.edge[k];
        const int x = (int)(c % a.nx);
        const int y = (int)((c / a.nx) % a.ny);
        const int z = (int)(c / a.nxy);
        S *p = static_cast<S *>(a.pdf);
        R *ub = static_cast<R *>(a.ub);
        const int64_t pl = 3 * ((int64_t)y + (int64_t)a.ny * z);
        R f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (ODD) {
                int64_t nbr = 0;
                const int kind = classify(a, x - cx_of(i), y - cy_of(i), z - cz_of(i), nbr);
                if (kind == LINK_FLUID) {
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
        const Rates rt{a.w1, a.w2, a.w3, a.galilean};
        collide<R, PLAIN>(f, rt, drho, ux, uy, uz);
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
            int64_t nbr = 0;
            const int kind = classify(a, x - cx_of(i), y - cy_of(i), z - cz_of(i), nbr);
            if (kind == LINK_SOLID) {   // momentum exchange with the obstacle
                fx += 2.0 * cx_of(j) * (double)f[j];
                fy += 2.0 * cy_of(j) * (double)f[j];
                fz += 2.0 * cz_of(j) * (double)f[j];
            }
            if (ODD) {
                if (kind == LINK_FLUID) {
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
    if (a.fpart) block_force_reduce(a, fx, fy, fz);
}

template <class S>
void launch_step_t(const StepArgs &a, bool odd, bool epi, bool plain, int block_x, cudaStream_t s, cudaEvent_t mid)
{
    const dim3 blk(block_x);
    const dim3 grd((a.nx + block_x - 1) / block_x, a.ny, a.nz);
#define LBM_BULK(O, E, P) k_step_bulk<S, O, E, P><<<grd, blk, 0, s>>>(a)
    if (plain) {
        if (odd) { if (epi) LBM_BULK(true, true, true); else LBM_BULK(true, false, true); }
        else     { if (epi) LBM_BULK(false, true, true); else LBM_BULK(false, false, true); }
    } else {
        if (odd) { if (epi) LBM_BULK(true, true, false); else LBM_BULK(true, false, false); }
        else     { if (epi) LBM_BULK(false, true, false); else LBM_BULK(false, false, false); }
    }
#undef LBM_BULK
    if (mid) cudaEventRecord(mid, s);
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
