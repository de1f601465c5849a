// lbm_aux.cu -- set-up and read-out kernels around the step: cell flags,
// seeded initial states, natural-order gathers of the AA state, macroscopic
// fields, time-average read-out, half-resolution box means and deterministic
// FP64 totals.
#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// cell flags: solid, or edge (some neighbour outside the domain or solid)
// ---------------------------------------------------------------------------
// Cell classes.  A fluid cell is an edge cell when it has an obstacle
// neighbour or one of its links crosses a periodic face (wrap-around).  A
// fluid cell whose boundary links all cross one x face (inlet/outlet planes)
// is an x-face cell, updated by the bulk kernel; one whose boundary links all
// cross no-slip lateral walls is a wall cell, updated by the wall-row blocks
// of the edge kernel.
// Where an x face meets a wall the cells stay edge cells, and so do the wall
// rows of a grid less than two cells wide in y or z (where the rows y = 0 and
// y = ny - 1, or z = 0 and z = nz - 1, coincide).
__global__ void k_flags(const uint8_t *mask, uint8_t *flags, int nx, int ny, int nz, int xface_lo, int xface_hi,
                        int wall_y, int wall_z)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
        if (mask && mask[c]) { flags[c] = CELL_SOLID; continue; }
        bool solid_nbr = false;
        if (mask) {
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int xx = x + dx, yy = y + dy, zz = z + dz;
                        if (xx < 0 || yy < 0 || zz < 0 || xx >= nx || yy >= ny || zz >= nz) continue;
                        if (mask[xx + (int64_t)nx * (yy + (int64_t)ny * zz)]) solid_nbr = true;
                    }
        }
        const bool y_face = y == 0 || y == ny - 1, z_face = z == 0 || z == nz - 1;
        const bool x_face = x == 0 || x == nx - 1;
        // every face a link of this cell crosses must be non-periodic; a grid
        // one cell thick in x has both x faces on one cell: edge kernel
        const bool x_ok = !x_face || (nx >= 2 && (x == 0 ? xface_lo : xface_hi));
        const bool w_ok = (!y_face || (wall_y && ny >= 2)) && (!z_face || (wall_z && nz >= 2));
        uint8_t fl = 0;
        if (solid_nbr || !x_ok || !w_ok || (x_face && (y_face || z_face))) fl = CELL_EDGE;
        else if (x_face) fl = CELL_XFACE;
        else if (y_face || z_face) fl = CELL_WALL;
        flags[c] = fl;
    }
}

void launch_flags(const uint8_t *mask, uint8_t *flags, int nx, int ny, int nz, bool xface_lo, bool xface_hi,
                  bool wall_y, bool wall_z, cudaStream_t s)
{
    k_flags<<<1216, 256, 0, s>>>(mask, flags, nx, ny, nz, xface_lo, xface_hi, wall_y, wall_z);
}


// ---------------------------------------------------------------------------
// Boundary-cell records, built on the device in two passes over fixed chunks
// of EB_CHUNK cells (one block each): the counts of every chunk, then, after
// an exclusive scan of the edge counts on the host, each chunk writes its
// records in ascending cell order at its offset (a block-wide ballot scan),
// so the list is the same whatever the scheduling.  The link codes follow
// the pull view of the step kernels: where population i of the cell comes
// from (x - c_i): a lateral face is a wall unless periodic; then the x
// faces (inlet, outlet or wall, or a wrap); then an obstacle cell.  Solid
// links are counted per direction j heading into the obstacle (integer
// atomics: exact and order-free) for the constant part of the force.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t record_link(const uint8_t *flags, int nx, int ny, int nz, int fxlo, int fxhi,
                                                int fy, int fz, int sx, int sy, int sz)
{
    bool wrapped = false;
    if (sy < 0 || sy >= ny) {
        if (fy != FACE_PERIODIC) return LINK_WALL;
        sy = sy < 0 ? sy + ny : sy - ny;
        wrapped = true;
    }
    if (sz < 0 || sz >= nz) {
        if (fz != FACE_PERIODIC) return LINK_WALL;
        sz = sz < 0 ? sz + nz : sz - nz;
        wrapped = true;
    }
    if (sx < 0) {
        if (fxlo == FACE_INLET) return LINK_INLET;
        if (fxlo == FACE_WALL) return LINK_WALL;
        sx += nx;
        wrapped = true;
    } else if (sx >= nx) {
        if (fxhi == FACE_OUTLET || fxhi == FACE_OUTFLOW) return LINK_OUTLET;
        if (fxhi == FACE_WALL) return LINK_WALL;
        sx -= nx;
        wrapped = true;
    }
    if (flags[sx + (int64_t)nx * (sy + (int64_t)ny * sz)] & CELL_SOLID) return LINK_SOLID;
    return wrapped ? LINK_WRAP : LINK_FLUID;
}

__global__ void __launch_bounds__(EB_THREADS) k_record_count(const uint8_t *flags, int64_t n, int *counts)
{
    __shared__ int sc[4];
    if (threadIdx.x < 4) sc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t c0 = (int64_t)blockIdx.x * EB_CHUNK;
    int v[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < EB_CHUNK; k += blockDim.x) {
        const int64_t c = c0 + k;
        if (c >= n) break;
        const uint8_t fl = flags[c];
        v[0] += !(fl & CELL_SOLID);
        v[1] += (fl == 0 || fl == CELL_XFACE);
        v[2] += fl == CELL_WALL;
        v[3] += fl == CELL_EDGE;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sc[q], v[q]);
    }
    __syncthreads();
    if (threadIdx.x < 4) counts[4 * blockIdx.x + threadIdx.x] = sc[threadIdx.x];
}

__global__ void __launch_bounds__(EB_THREADS) k_record_write(const uint8_t *flags, int nx, int ny, int nz, int fxlo,
                                                             int fxhi, int fy, int fz, const int64_t *offsets,
                                                             uint4 *edge, unsigned long long *solid)
{
    __shared__ int wt[EB_THREADS / 32];
    const int64_t n = (int64_t)nx * ny * nz;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t base = offsets[blockIdx.x];
    const int64_t c0 = (int64_t)blockIdx.x * EB_CHUNK;
    for (int k0 = 0; k0 < EB_CHUNK; k0 += EB_THREADS) {
        const int64_t c = c0 + k0 + threadIdx.x;
        const bool rec = c < n && flags[c] == CELL_EDGE;
        const unsigned bal = __ballot_sync(0xffffffffu, rec);
        if (lane == 0) wt[wid] = __popc(bal);
        __syncthreads();
        int before = 0, total = 0;
#pragma unroll
        for (int q = 0; q < EB_THREADS / 32; ++q) {
            before += q < wid ? wt[q] : 0;
            total += wt[q];
        }
        if (rec) {
            const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((int64_t)nx * ny));
            uint32_t w[3] = {0u, 0u, 0u};
            for (int i = 0; i < Q; ++i) {
                const uint32_t kind = record_link(flags, nx, ny, nz, fxlo, fxhi, fy, fz, x - cx_of(i), y - cy_of(i),
                                                  z - cz_of(i));
                w[i / 9] |= kind << (3 * (i % 9));
                if (kind == LINK_SOLID) atomicAdd(&solid[Q - 1 - i], 1ull);
            }
            edge[base + before + __popc(bal & ((1u << lane) - 1u))] = make_uint4((uint32_t)c, w[0], w[1], w[2]);
        }
        base += total;
        __syncthreads();
    }
}

__global__ void k_gather_flags(const uint8_t *flags, const int64_t *idx, int64_t m, uint8_t *out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = flags[idx[k]];
}

void launch_gather_flags(const uint8_t *flags, const int64_t *idx, int64_t m, uint8_t *out, cudaStream_t s)
{
    k_gather_flags<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, s>>>(flags, idx, m, out);
}

int64_t record_blocks(int64_t n) { return (n + EB_CHUNK - 1) / EB_CHUNK; }

void launch_record_count(const uint8_t *flags, int64_t n, int *counts, cudaStream_t s)
{
    k_record_count<<<(unsigned)record_blocks(n), EB_THREADS, 0, s>>>(flags, n, counts);
}

void launch_record_write(const uint8_t *flags, int nx, int ny, int nz, int fxlo, int fxhi, int fy, int fz,
                         const int64_t *offsets, uint4 *edge, unsigned long long *solid, cudaStream_t s)
{
    k_record_write<<<(unsigned)record_blocks((int64_t)nx * ny * nz), EB_THREADS, 0, s>>>(
        flags, nx, ny, nz, fxlo, fxhi, fy, fz, offsets, edge, solid);
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014; Vigna's reference constants):
// output `ctr` of the stream started at `seed` is mix(seed + (ctr+1) golden).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t ctr)
{
    uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class S>
__global__ void k_noise(S *pdf, int64_t slot, const uint8_t *flags, int64_t n, uint64_t seed, double amp)
{
    using T = Store<S>;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const bool solid = flags[c] & CELL_SOLID;
        for (int i = 0; i < Q; ++i) {
            double v = 0.0;
            if (!solid) {
                const uint64_t z = splitmix64(seed, (uint64_t)c * Q + i);
                const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
                v = amp * (2.0 * u - 1.0);
            }
            T::st(pdf + i * slot + c, (typename T::R)v);
        }
    }
}

// ---------------------------------------------------------------------------
// natural-order populations of the current state (FP64, shifted)
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ void gather_natural(const StepArgs &a, bool odd, int64_t c, double *f)
{
    using T = Store<S>;
    using R = typename T::R;
    const S *p = static_cast<const S *>(a.pdf);
    if (!odd) {
        for (int i = 0; i < Q; ++i) f[i] = (double)T::ld(p + (int64_t)i * a.slot + c);
        return;
    }
    const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny), z = (int)(c / a.nxy);
    const R *ub = static_cast<const R *>(a.ub);
    const int64_t pl = 3 * ((int64_t)y + (int64_t)a.ny * z);
    for (int i = 0; i < Q; ++i) {
        int64_t nbr = 0;
        const int kind = classify(a, x - cx_of(i), y - cy_of(i), z - cz_of(i), nbr);
        if (kind == LINK_FLUID) {
            f[i] = (double)T::ld(p + (int64_t)(Q - 1 - i) * a.slot + nbr);
        } else {
            const double own = (double)T::ld(p + (int64_t)i * a.slot + c);
            if (kind == LINK_OUTLET)
                f[i] = boundary_value<double>(a, kind, i, own, (double)ub[pl], (double)ub[pl + 1], (double)ub[pl + 2]);
            else
                f[i] = boundary_value<double>(a, kind, i, own, 0.0, 0.0, 0.0);
        }
    }
}

// out[i * si + k * sc] = w_i + fbar_i of cell cells[k] (or cell k when cells is null)
template <class S>
__global__ void k_gather(StepArgs a, bool odd, const int64_t *cells, int64_t count, double *out, int64_t si, int64_t sc)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cells ? cells[k] : k;
        double f[Q];
        if (c < 0 || c >= a.n) {            // out-of-range request: NaN, no access
            for (int i = 0; i < Q; ++i) out[i * si + k * sc] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        if (a.flags[c] & CELL_SOLID) {
            for (int i = 0; i < Q; ++i) f[i] = 0.0;
        } else {
            gather_natural<S>(a, odd, c, f);
        }
        for (int i = 0; i < Q; ++i) out[i * si + k * sc] = w_of(i) + f[i];
    }
}

template <class S>
__global__ void k_set(S *pdf, int64_t slot, const uint8_t *flags, int64_t n, const double *src)
{
    using T = Store<S>;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const bool solid = flags[c] & CELL_SOLID;
        for (int i = 0; i < Q; ++i)
            T::st(pdf + i * slot + c, (typename T::R)(solid ? 0.0 : src[i * n + c] - w_of(i)));
    }
}

// Populations at the product-form equilibrium of given fields, per cell
// (ux, uy, uz, p), rho = 1 + 3 p: f_i = rho phi(cx, ux) phi(cy, uy) phi(cz, uz)
// with phi(0, u) = 2/3 - u^2 and phi(+-1, u) = (1/3 + u^2 +- u)/2 (the
// equilibrium whose cumulants above second order vanish); stored shifted,
// solid cells at rest.  FP64 arithmetic.
__device__ __forceinline__ double eq_phi(int c, double u)
{
    return c == 0 ? 2.0 / 3.0 - u * u : 0.5 * (1.0 / 3.0 + u * u + c * u);
}

template <class S>
__global__ void k_equilibrium(S *pdf, int64_t slot, const uint8_t *flags, int64_t n, const float *fields)
{
    using T = Store<S>;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const bool solid = flags[c] & CELL_SOLID;
        const float4 v = reinterpret_cast<const float4 *>(fields)[c];
        const double ux = v.x, uy = v.y, uz = v.z, rho = 1.0 + 3.0 * (double)v.w;
        for (int i = 0; i < Q; ++i) {
            const double f = rho * eq_phi(cx_of(i), ux) * eq_phi(cy_of(i), uy) * eq_phi(cz_of(i), uz);
            T::st(pdf + i * slot + c, (typename T::R)(solid ? 0.0 : f - w_of(i)));
        }
    }
}

template <class S>
__global__ void k_macros(StepArgs a, bool odd, double *rho, double *u)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < a.n; c += (int64_t)gridDim.x * blockDim.x) {
        if (a.flags[c] & CELL_SOLID) {
            rho[c] = 1.0;
            u[3 * c] = u[3 * c + 1] = u[3 * c + 2] = 0.0;
            continue;
        }
        double f[Q];
        gather_natural<S>(a, odd, c, f);
        double d = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < Q; ++i) {
            d += f[i];
            jx += cx_of(i) * f[i];
            jy += cy_of(i) * f[i];
            jz += cz_of(i) * f[i];
        }
        const double r = 1.0 + d;
        rho[c] = r;
        u[3 * c] = jx / r;
        u[3 * c + 1] = jy / r;
        u[3 * c + 2] = jz / r;
    }
}

// Per-block partial totals (mass deviation, momentum) in fixed order; the
// second kernel adds the partials in fixed order.
constexpr int TOT_BLOCK = 256;

template <class S>
__global__ void __launch_bounds__(TOT_BLOCK) k_totals_partial(StepArgs a, bool odd, double *partials)
{
    __shared__ double sh[4][TOT_BLOCK];
    double acc[4] = {0, 0, 0, 0};
    for (int64_t c = (int64_t)blockIdx.x * TOT_BLOCK + threadIdx.x; c < a.n; c += (int64_t)gridDim.x * TOT_BLOCK) {
        if (a.flags[c] & CELL_SOLID) continue;
        double f[Q];
        gather_natural<S>(a, odd, c, f);
        for (int i = 0; i < Q; ++i) {
            acc[0] += f[i];
            acc[1] += cx_of(i) * f[i];
            acc[2] += cy_of(i) * f[i];
            acc[3] += cz_of(i) * f[i];
        }
    }
    for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int h = TOT_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 4; ++d) partials[4 * (int64_t)blockIdx.x + d] = sh[d][0];
}

__global__ void __launch_bounds__(TOT_BLOCK) k_totals_final(const double *partials, int nblocks, double *out)
{
    __shared__ double sh[4][TOT_BLOCK];
    double acc[4] = {0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += TOT_BLOCK)
        for (int d = 0; d < 4; ++d) acc[d] += partials[4 * (int64_t)b + d];
    for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] = acc[d];
    __syncthreads();
    for (int h = TOT_BLOCK / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int d = 0; d < 4; ++d) sh[d][threadIdx.x] += sh[d][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 4; ++d) out[d] = sh[d][0];
}

// ---------------------------------------------------------------------------
// time average read-out: (ux, uy, uz, p) per cell from the FP64 sums
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_mean_out(const double *msum, int64_t n, double inv_samples, T *out)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        out[4 * c + 0] = (T)(msum[n + c] * inv_samples);
        out[4 * c + 1] = (T)(msum[2 * n + c] * inv_samples);
        out[4 * c + 2] = (T)(msum[3 * n + c] * inv_samples);
        out[4 * c + 3] = (T)(msum[c] * inv_samples * (1.0 / 3.0));
    }
}

// Velocity covariances from the running sums: msum [4][n] means then [6][n]
// products (xx, yy, zz, xy, xz, yz) -> out [n][6].
template <class T>
__global__ void k_stats_out(const double *msum, int64_t n, double inv_samples, T *out)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double mx = msum[n + c] * inv_samples, my = msum[2 * n + c] * inv_samples,
                     mz = msum[3 * n + c] * inv_samples;
        const double *q = msum + 4 * n + c;
        out[6 * c + 0] = (T)(q[0] * inv_samples - mx * mx);
        out[6 * c + 1] = (T)(q[n] * inv_samples - my * my);
        out[6 * c + 2] = (T)(q[2 * n] * inv_samples - mz * mz);
        out[6 * c + 3] = (T)(q[3 * n] * inv_samples - mx * my);
        out[6 * c + 4] = (T)(q[4 * n] * inv_samples - mx * mz);
        out[6 * c + 5] = (T)(q[5 * n] * inv_samples - my * mz);
    }
}

// 2x2x2 box mean of a [z][y][x][4] field; a trailing odd cell is a block of its own.
template <class T>
__global__ void k_halfres(const T *in, int nx, int ny, int nz, T *out)
{
    const int hx = (nx + 1) / 2, hy = (ny + 1) / 2, hz = (nz + 1) / 2;
    const int64_t nh = (int64_t)hx * hy * hz;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(h % hx), Y = (int)((h / hx) % hy), Z = (int)(h / ((int64_t)hx * hy));
        double s[4] = {0, 0, 0, 0};
        int cnt = 0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
                    if (x >= nx || y >= ny || z >= nz) continue;
                    const int64_t c = x + (int64_t)nx * (y + (int64_t)ny * z);
                    for (int d = 0; d < 4; ++d) s[d] += (double)in[4 * c + d];
                    ++cnt;
                }
        for (int d = 0; d < 4; ++d) out[4 * h + d] = (T)(s[d] / cnt);
    }
}

// (ux, uy, uz, p) of the current state at cell c (p = (rho - 1)/3; solid or
// out-of-range cells give 0).
template <class S>
__device__ __forceinline__ float4 cell_macros(const StepArgs &a, bool odd, int64_t c)
{
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c >= 0 && c < a.n && !(a.flags[c] & CELL_SOLID)) {
        double f[Q];
        gather_natural<S>(a, odd, c, f);
        double d = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < Q; ++i) {
            d += f[i];
            jx += cx_of(i) * f[i];
            jy += cy_of(i) * f[i];
            jz += cz_of(i) * f[i];
        }
        const double r = 1.0 + d;
        v = make_float4((float)(jx / r), (float)(jy / r), (float)(jz / r), (float)(d / 3.0));
    }
    return v;
}

// Probe row: (ux, uy, uz, p) of the current state at the listed cells.
template <class S>
__global__ void k_probe(StepArgs a, bool odd, const int64_t *cells, int64_t count, float *out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<float4 *>(out)[k] = cell_macros<S>(a, odd, cells[k]);
}

// Monitor plane (Sec. 2: 2D snapshots of the centre x-y plane): (ux, uy, uz,
// p) of every cell of the plane z = z0 of the current state, [y][x] float4;
// consecutive threads take consecutive x.
template <class S>
__global__ void k_plane(StepArgs a, bool odd, int z0, float *out)
{
    const int64_t m = a.nxy, base = a.nxy * z0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<float4 *>(out)[k] = cell_macros<S>(a, odd, base + k);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int block) { return (int)std::min<int64_t>((n + block - 1) / block, gb300::sm_count() * 32); }

template <class S>
static void launch_aux_t(AuxOp op, const StepArgs &a, bool odd, const AuxArgs &x, cudaStream_t s)
{
    switch (op) {
    case AUX_NOISE:
        k_noise<S><<<grid_for(a.n, 256), 256, 0, s>>>((S *)a.pdf, a.slot, a.flags, a.n, x.seed, x.amp);
        break;
    case AUX_GATHER:
        k_gather<S><<<grid_for(x.count, 128), 128, 0, s>>>(a, odd, x.cells, x.count, x.out, x.si, x.sc);
        break;
    case AUX_SET:
        k_set<S><<<grid_for(a.n, 256), 256, 0, s>>>((S *)a.pdf, a.slot, a.flags, a.n, x.src);
        break;
    case AUX_MACROS:
        k_macros<S><<<grid_for(a.n, 128), 128, 0, s>>>(a, odd, x.out, x.out2);
        break;
    case AUX_TOTALS:
        k_totals_partial<S><<<x.nblocks, TOT_BLOCK, 0, s>>>(a, odd, x.partials);
        k_totals_final<<<1, TOT_BLOCK, 0, s>>>(x.partials, x.nblocks, x.out);
        break;
    case AUX_PROBE:
        k_probe<S><<<grid_for(x.count, 128), 128, 0, s>>>(a, odd, x.cells, x.count, x.fout);
        break;
    case AUX_PLANE:
        k_plane<S><<<grid_for(a.nxy, 128), 128, 0, s>>>(a, odd, (int)x.count, x.fout);
        break;
    case AUX_EQUILIBRIUM:
        k_equilibrium<S><<<grid_for(a.n, 256), 256, 0, s>>>((S *)a.pdf, a.slot, a.flags, a.n, x.fsrc);
        break;
    }
}

void launch_aux(int storage, AuxOp op, const StepArgs &a, bool odd, const AuxArgs &x, cudaStream_t s)
{
    switch (storage) {
    case 0: launch_aux_t<double>(op, a, odd, x, s); break;
    case 1: launch_aux_t<float>(op, a, odd, x, s); break;
    case 2: launch_aux_t<__half>(op, a, odd, x, s); break;
    case 3: launch_aux_t<__nv_bfloat16>(op, a, odd, x, s); break;
    default: launch_aux_t<F16C>(op, a, odd, x, s); break;
    }
}

void launch_mean_out(const double *msum, int64_t n, double inv_samples, bool f32, void *out, cudaStream_t s)
{
    if (f32) k_mean_out<float><<<grid_for(n, 256), 256, 0, s>>>(msum, n, inv_samples, (float *)out);
    else k_mean_out<double><<<grid_for(n, 256), 256, 0, s>>>(msum, n, inv_samples, (double *)out);
}

void launch_stats_out(const double *msum, int64_t n, double inv_samples, bool f32, void *out, cudaStream_t s)
{
    if (f32) k_stats_out<float><<<grid_for(n, 256), 256, 0, s>>>(msum, n, inv_samples, (float *)out);
    else k_stats_out<double><<<grid_for(n, 256), 256, 0, s>>>(msum, n, inv_samples, (double *)out);
}

// FP32 snapshot box mean: one thread per half-resolution cell, 16-byte loads
// of the (u, v, w, p) records (consecutive threads read consecutive pairs).
__global__ void k_halfres_f4(const float4 *in, int nx, int ny, int nz, float4 *out)
{
    const int hx = (nx + 1) / 2, hy = (ny + 1) / 2, hz = (nz + 1) / 2;
    const int64_t nh = (int64_t)hx * hy * hz;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(h % hx), Y = (int)((h / hx) % hy), Z = (int)(h / ((int64_t)hx * hy));
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        int cnt = 0;
        for (int dz = 0; dz < 2; ++dz) {
            const int z = 2 * Z + dz;
            if (z >= nz) continue;
            for (int dy = 0; dy < 2; ++dy) {
                const int y = 2 * Y + dy;
                if (y >= ny) continue;
                const int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
                for (int dx = 0; dx < 2; ++dx) {
                    const int x = 2 * X + dx;
                    if (x >= nx) continue;
                    const float4 v = in[row + x];
                    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
                    ++cnt;
                }
            }
        }
        const float r = 1.0f / (float)cnt;
        out[h] = make_float4(acc.x * r, acc.y * r, acc.z * r, acc.w * r);
    }
}

void launch_halfres(const void *in, int nx, int ny, int nz, bool f32, void *out, cudaStream_t s)
{
    const int64_t nh = (int64_t)((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2);
    if (f32) k_halfres_f4<<<grid_for(nh, 256), 256, 0, s>>>((const float4 *)in, nx, ny, nz, (float4 *)out);
    else k_halfres<double><<<grid_for(nh, 256), 256, 0, s>>>((const double *)in, nx, ny, nz, (double *)out);
}

}  // namespace lbm
