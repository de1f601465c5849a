// lbm_device.cuh -- device-side building blocks of the D3Q27 cumulant step:
// storage traits, link classification, the shifted-form chimera transform
// and the cumulant collision (Sec. 3.2 of the paper: D3Q27 stencil and
// cumulant collision operator; relaxation after Geier et al. 2015, cited there).
//
// Populations are stored shifted, fbar_i = f_i - w_i, and every step of the
// collision works on deviations from the rest state so that FP32 arithmetic
// keeps the small hydrodynamic signal (|fbar| ~ 1e-2) instead of rounding it
// against the O(1) weights.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 27;
// threads per block of the edge-cell kernel (also sizes the force partials)
constexpr int EDGE_BLOCK = 128;
// threads per wall-row block of the edge kernel (one row segment of cells along x)
constexpr int WALL_BLOCK = 128;

// Velocity components of direction i = (cx+1) + 3(cy+1) + 9(cz+1).
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }
// 1-D weight factors t(c): 2/3 at rest, 1/6 for +-1; w_i = t(cx) t(cy) t(cz).
__host__ __device__ constexpr double tw(int k) { return k == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double w_of(int i) { return tw(i % 3) * tw((i / 3) % 3) * tw(i / 9); }
// Moments of t about the mean in one dimension: order 0 -> 1, 1 -> 0, 2 -> 1/3.
__host__ __device__ constexpr double zw(int a) { return a == 0 ? 1.0 : (a == 1 ? 0.0 : 1.0 / 3.0); }

// cell classes: solid; edge (boundary-aware kernel); x-face (an inlet or
// outlet plane cell whose only boundary links cross that x face; handled by
// the row-end variant of the bulk kernel); wall (a cell in a row next to a
// no-slip lateral wall whose only boundary links cross that wall; handled by
// the wall-row blocks of the edge kernel); 0 = bulk
enum : uint8_t { CELL_SOLID = 1, CELL_EDGE = 2, CELL_XFACE = 4, CELL_WALL = 8 };
// Rows (y, z) next to a lateral wall, numbered y = 0 (nz rows), y = ny - 1
// (nz rows), then z = 0 and z = nz - 1 for 0 < y < ny - 1 (ny - 2 rows each):
// distinct rows when ny, nz >= 2 (wall cells exist only then).
__host__ __device__ constexpr int64_t wall_rows(int ny, int nz)
{
    return 2 * (int64_t)nz + 2 * (int64_t)(ny > 2 ? ny - 2 : 0);
}
__host__ __device__ inline void wall_row_yz(int64_t r, int ny, int nz, int &y, int &z)
{
    if (r < nz) { y = 0; z = (int)r; return; }
    if (r < 2 * (int64_t)nz) { y = ny - 1; z = (int)(r - nz); return; }
    const int64_t k = r - 2 * (int64_t)nz, m = ny - 2;
    if (k < m) { z = 0; y = 1 + (int)k; return; }
    z = nz - 1; y = 1 + (int)(k - m);
}

// face kinds (lbm_face): x high is either the anti-bounce-back pressure
// outlet or the convective extrapolation outflow
enum { FACE_WALL = 0, FACE_PERIODIC = 1, FACE_INLET = 2, FACE_OUTLET = 3, FACE_OUTFLOW = 4 };
// link kinds of the cell a population comes from (pull view); LINK_WRAP is a
// fluid neighbour reached through a periodic face
enum { LINK_FLUID = 0, LINK_WALL = 1, LINK_SOLID = 2, LINK_INLET = 3, LINK_OUTLET = 4, LINK_WRAP = 5 };
// device status bits
enum { STATUS_UNSTABLE = 1 };

// ---------------------------------------------------------------------------
// storage traits
// ---------------------------------------------------------------------------
template <class S> struct Store;
template <> struct Store<double> {
    using R = double;
    static __device__ __forceinline__ double ld(const double *p) { return *p; }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Store<float> {
    using R = float;
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Store<__half> {
    using R = float;
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<__nv_bfloat16> {
    using R = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};

// 16-bit custom float for shifted populations: sign, 4 exponent bits (bias
// 15), 11 mantissa bits; normal range 2^-14 .. 2 - 2^-11, subnormal step
// 2^-25.  Shifted populations of a stable flow stay well inside (-1, 1), so
// one exponent bit of IEEE binary16 is traded for one more mantissa bit.
// The code is the FP32 pattern of v 2^-112 with its 12 low mantissa bits
// dropped: the FP32 exponent field of v 2^-112 is then the 4-bit field.
//   decode: the code loaded sign-extended and shifted left by 12 puts the sign
//     on bit 31 and the 15 magnitude bits on bits 12..26 (bits 27..30, copies
//     of the sign, are masked off); times 2^112.  Two integer operations.
//   encode: clamp to the largest code (NaN too), scale by 2^-112, round the
//     dropped bits to nearest (ties away from zero: add half a unit of the
//     12th bit to the magnitude), keep bits 12..26 and the sign.
struct F16C {
    uint16_t bits;
};
template <> struct Store<F16C> {
    using R = float;
    static constexpr float MAXV = 1.99951171875f;   // 2 - 2^-11
    static __device__ __forceinline__ float ld(const F16C *p)
    {
        const int32_t b = (int32_t)(*reinterpret_cast<const int16_t *>(p));
        return __uint_as_float(((uint32_t)b << 12) & 0x87FFF000u) * 0x1p112f;
    }
    static __device__ __forceinline__ void st(F16C *p, float v)
    {
        v = fminf(fmaxf(v, -MAXV), MAXV);
        const uint32_t u = __float_as_uint(v * 0x1p-112f);
        const uint32_t r = u + 0x800u;
        p->bits = (uint16_t)((r >> 12) | ((u >> 16) & 0x8000u));
    }
};

// ---------------------------------------------------------------------------
// launch arguments shared by the step kernels (plain data, passed by value)
// ---------------------------------------------------------------------------
struct StepArgs {
    void *pdf;              // 27 slots of `slot` elements each
    int64_t slot;
    const uint8_t *flags;   // per cell: CELL_SOLID / CELL_EDGE
    const uint4 *edge;      // edge-cell records {cell, link codes 0-8, 9-17, 18-26}
    int64_t n_edge;
    int nx, ny, nz;
    int64_t nxy, n;
    double w1, w2, w3;      // shear, bulk, higher-order rates
    int galilean;
    // fourth-order parametrisation (param4 != 0): omega3, omega4, omega5,
    // the fourth-order factors -(2/3) A (1/w1 - 1/2) and B (1 - w1/2), and
    // the limiter lambda (p4) with their FP32 copies (p4f)
    int param4;
    double p4[6];
    float p4f[6];
    int xface_bulk;         // 1: the bulk kernel updates the inlet/outlet cells in its face warps
    int face_x_lo, face_x_hi, face_y, face_z;
    double u_in, rho_in, rho_out;
    // FP32 copies of the rates and boundary constants, so that FP32 kernels
    // never touch the FP64 pipe
    float w1f, w2f, w3f, u_in_f, rho_in_f, rho_out_f;
    // byte offsets of the bulk accesses relative to the cell's slot-0 address:
    // index 0/1 = even gather/scatter, 2/3 = odd gather/scatter
    int64_t boff[4][27];
    void *ub;               // outlet plane velocity [nz*ny][3] (compute type)
    void *ob;               // outflow planes (compute type): [9][nz*ny] pre-collision
                            // populations with cx = -1 of the outlet cells, then
                            // [9][nz*ny] of the cells next to them (x = nx - 2),
                            // recorded between steps by k_outflow
    double *msum;           // mean sums [4][n] (+ [6][n] velocity products when
                            // `stats`) when this step is sampled, else null
    int stats;              // accumulate velocity products with the means
    // interpolated bounce-back on obstacle links (after the step, k_qbb):
    // records {cell, x1 = cell + c_i, x2 = cell + 2 c_i, i | mode << 8} with i
    // the returning (pull) direction, mode 1 linear / 2 quadratic; q per link
    const uint4 *qlinks;
    const double *qval;
    int64_t n_qlinks;
    double *qpart;          // force partials per q-link block
    unsigned int *qcount;   // arrival counter of that reduction
    float *snap;            // full-resolution float4 target when snapshotting, else null
    double *fpart;          // force partials per edge block when recorded, else null
    unsigned int *fcount;   // arrival counter of the last-block reduction
    double *fout;           // force row of this step (3 doubles)
    int *status;            // latched device conditions
    int64_t n_wall;         // cells of class CELL_WALL (0: no wall-row blocks)
};

// Member of a batched launch (device memory): the static arguments of the
// member lattice plus its schedule.
struct BatchMember {
    StepArgs a;             // static fields (msum/snap/fout of `a` unused)
    double *msum;           // mean sums (null: no time average)
    int64_t mean_start, mean_end, mean_every;
    double *force;          // force rows indexed by t / force_every (null: off)
    int64_t force_every;
    int32_t gx, gy;         // bulk blocks along x and y per z plane
    int32_t wx;             // wall-row blocks along x (WALL_BLOCK cells each)
};

// One batched step: device member table and block numbering.
struct BatchLaunch {
    const BatchMember *mem;
    const int64_t *bulk_begin;  // nm + 1 entries (first bulk block per member)
    const int64_t *edge_begin;  // nm + 1 entries (first edge block per member)
    int nm;
    int64_t bulk_blocks, edge_blocks;
    int64_t *t;                 // device step counter
    int block_x, block_y;
    int out_chunks;             // outflow: blocks per member along its outlet plane (0: none)
    const int64_t *q_begin;     // nm + 1 entries (first wall-distance block per member)
    int64_t q_blocks;           // wall-distance blocks in all (0: none)
    const int64_t *w_begin;     // nm + 1 entries (first wall-row block per member)
    int64_t w_blocks;           // wall-row blocks in all (0: none)
};

// A parameter in the compute type: the FP32 copy for float kernels.
template <class R> __device__ __forceinline__ R pick(double d, float f);
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }

// ---------------------------------------------------------------------------
// link classification (Sec. 3.1: velocity inlet, outflow, no-slip lateral
// walls; obstacle cells bounce back).  A link that leaves through y or z is a
// wall link even when it also crosses x; then x; then obstacle cells.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int classify(const StepArgs &a, int sx, int sy, int sz, int64_t &nbr)
{
    if (sy < 0 || sy >= a.ny) {
        if (a.face_y != FACE_PERIODIC) return LINK_WALL;
        sy = sy < 0 ? sy + a.ny : sy - a.ny;
    }
    if (sz < 0 || sz >= a.nz) {
        if (a.face_z != FACE_PERIODIC) return LINK_WALL;
        sz = sz < 0 ? sz + a.nz : sz - a.nz;
    }
    if (sx < 0) {
        if (a.face_x_lo == FACE_INLET) return LINK_INLET;
        if (a.face_x_lo == FACE_WALL) return LINK_WALL;
        sx += a.nx;
    } else if (sx >= a.nx) {
        if (a.face_x_hi == FACE_OUTLET || a.face_x_hi == FACE_OUTFLOW) return LINK_OUTLET;
        if (a.face_x_hi == FACE_WALL) return LINK_WALL;
        sx -= a.nx;
    }
    nbr = (int64_t)sx + (int64_t)a.nx * ((int64_t)sy + (int64_t)a.ny * sz);
    return (a.flags[nbr] & CELL_SOLID) ? LINK_SOLID : LINK_FLUID;
}

// Shifted value delivered through a boundary link into direction i of a cell
// whose own slot holds `own` (the post-collision population of the opposite
// direction).  Halfway bounce-back for walls and obstacles, bounce-back from
// a wall moving with (u_in, 0, 0) at the inlet, anti-bounce-back against the
// even part of the equilibrium at rho_out with velocity ub at the pressure
// outlet.  With the convective outflow the own slot already holds the
// extrapolated value (written after the previous step by k_outflow).
// Rounded add and multiply that the compiler does not fuse.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <class R>
__device__ __forceinline__ R boundary_value(const StepArgs &a, int kind, int i, R own, R ubx, R uby, R ubz)
{
    const R w = R(w_of(i));
    // the inlet term with explicitly rounded operations: the same value in
    // every kernel that applies it (no contraction left to the compiler)
    if (kind == LINK_INLET)
        return add_rn(own, mul_rn(mul_rn(R(6) * w, pick<R>(a.rho_in, a.rho_in_f)),
                                  R(cx_of(i)) * pick<R>(a.u_in, a.u_in_f)));
    if (kind == LINK_OUTLET && a.face_x_hi == FACE_OUTFLOW) return own;
    if (kind == LINK_OUTLET) {
        const R cu = R(cx_of(i)) * ubx + R(cy_of(i)) * uby + R(cz_of(i)) * ubz;
        const R uu = ubx * ubx + uby * uby + ubz * ubz;
        // shifted form: -(own + w) + 2 w rho_out (1 + 4.5 cu^2 - 1.5 uu) - w
        return -own + R(2) * w * (pick<R>(a.rho_out, a.rho_out_f) * (R(1) + R(4.5) * cu * cu - R(1.5) * uu) - R(1));
    }
    return own;
}

// ---------------------------------------------------------------------------
// chimera line transforms in shifted form.  A line holds (f-, f0, f+) whose
// rest values are (K/6, 2K/3, K/6); the outputs are the zeroth moment minus K,
// the first central moment, and the second central moment minus K/3.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void fwd_line(R &a, R &b, R &c, R u, R K)
{
    const R s = c + a, d = c - a;
    const R m0 = s + b;
    const R mk = m0 + K;
    const R m1 = d - u * mk;
    const R m2 = s - R(2) * u * d + u * u * mk;
    a = m0;
    b = m1;
    c = m2;
}

// Inverse line transform through the line's raw moments: s1 = f+ - f- (first
// raw moment) and s2 = f+ + f- - K/3 (second raw moment, shifted).  Then
// f- = (s2 - s1)/2, f+ = (s2 + s1)/2, f0 = m0 - s2, so the zeroth moment is
// reproduced up to the rounding of the small deviation m0 (not of K).
template <class R>
__device__ __forceinline__ void inv_line(R &a, R &b, R &c, R u, R K)
{
    const R m0 = a, m1 = b, m2 = c;
    const R s1 = m1 + u * (m0 + K);
    const R s2 = m2 + u * (m1 + s1);
    a = R(0.5) * (s2 - s1);
    c = R(0.5) * (s2 + s1);
    b = m0 - s2;
}

#define MI(a, b, c) ((a) + 3 * (b) + 9 * (c))

// Forward chimera: populations (index (cx+1)+3(cy+1)+9(cz+1)) -> central
// moment deviations m[a + 3b + 9c] = kappa_abc - zw(a) zw(b) zw(c).
template <class R>
__device__ __forceinline__ void chimera_forward(R *f, R ux, R uy, R uz)
{
#pragma unroll
    for (int yi = 0; yi < 3; ++yi)
#pragma unroll
        for (int xi = 0; xi < 3; ++xi)
            fwd_line<R>(f[xi + 3 * yi], f[xi + 3 * yi + 9], f[xi + 3 * yi + 18], uz, R(tw(xi) * tw(yi)));
#pragma unroll
    for (int az = 0; az < 3; ++az)
#pragma unroll
        for (int xi = 0; xi < 3; ++xi)
            fwd_line<R>(f[xi + 9 * az], f[xi + 3 + 9 * az], f[xi + 6 + 9 * az], uy, R(tw(xi) * zw(az)));
#pragma unroll
    for (int az = 0; az < 3; ++az)
#pragma unroll
        for (int ay = 0; ay < 3; ++ay)
            fwd_line<R>(f[3 * ay + 9 * az], f[1 + 3 * ay + 9 * az], f[2 + 3 * ay + 9 * az], ux, R(zw(ay) * zw(az)));
}

template <class R>
__device__ __forceinline__ void chimera_inverse(R *f, R ux, R uy, R uz)
{
#pragma unroll
    for (int az = 0; az < 3; ++az)
#pragma unroll
        for (int ay = 0; ay < 3; ++ay)
            inv_line<R>(f[3 * ay + 9 * az], f[1 + 3 * ay + 9 * az], f[2 + 3 * ay + 9 * az], ux, R(zw(ay) * zw(az)));
#pragma unroll
    for (int az = 0; az < 3; ++az)
#pragma unroll
        for (int xi = 0; xi < 3; ++xi)
            inv_line<R>(f[xi + 9 * az], f[xi + 3 + 9 * az], f[xi + 6 + 9 * az], uy, R(tw(xi) * zw(az)));
#pragma unroll
    for (int yi = 0; yi < 3; ++yi)
#pragma unroll
        for (int xi = 0; xi < 3; ++xi)
            inv_line<R>(f[xi + 3 * yi], f[xi + 3 * yi + 9], f[xi + 3 * yi + 18], uz, R(tw(xi) * tw(yi)));
}

// Inverse line transform of a line whose first central moment is zero
// (m1 = 0): the lines (ay, az) with ay + az even of the x pass when every odd
// cumulant is zero after the collision.
template <class R>
__device__ __forceinline__ void inv_line_even(R &a, R &b, R &c, R u, R K)
{
    const R m0 = a, m2 = c;
    const R s1 = u * (m0 + K);
    const R s2 = m2 + u * s1;
    a = R(0.5) * (s2 - s1);
    c = R(0.5) * (s2 + s1);
    b = m0 - s2;
}

// Inverse line transform of a line holding only a first central moment
// (m0 = m2 = 0 and no rest part, K = 0): s1 = m1, s2 = 2 u m1, hence
// f- = m1 (u - 1/2), f+ = m1 (u + 1/2), f0 = -2 u m1.
template <class R>
__device__ __forceinline__ void inv_line_odd(R &a, R &b, R &c, R m1, R u_lo, R u_hi, R m2u)
{
    a = m1 * u_lo;
    c = m1 * u_hi;
    b = m1 * m2u;
}

// Inverse chimera after a collision that leaves every odd-order central
// moment zero (orders 1, 3, 5: every cumulant of order >= 3 reset).  The
// x pass then splits into lines with m1 = 0 ((ay, az) with ay + az even) and
// lines holding only m1 (ay + az odd, where the rest part K is zero too);
// the y and z passes are the general ones.  Arguments are the nonzero
// (non-normalised, deviation) central moments.
template <class R>
__device__ __forceinline__ void chimera_inverse_even(R *f, R ux, R uy, R uz, R m000, R m200, R m020, R m002, R m110,
                                                     R m101, R m011, R m211, R m121, R m112, R m220, R m202, R m022,
                                                     R m222)
{
    const R third = R(1.0 / 3.0), ninth = R(1.0 / 9.0);
    // x pass: line (ay, az) holds (m[0 ay az], m[1 ay az], m[2 ay az]) at
    // f[3 ay + 9 az + 0..2]
    f[0] = m000; f[2] = m200; inv_line_even<R>(f[0], f[1], f[2], ux, R(1));            // (0, 0)
    f[6] = m020; f[8] = m220; inv_line_even<R>(f[6], f[7], f[8], ux, third);           // (2, 0)
    f[12] = m011; f[14] = m211; inv_line_even<R>(f[12], f[13], f[14], ux, R(0));       // (1, 1)
    f[18] = m002; f[20] = m202; inv_line_even<R>(f[18], f[19], f[20], ux, third);      // (0, 2)
    f[24] = m022; f[26] = m222; inv_line_even<R>(f[24], f[25], f[26], ux, ninth);      // (2, 2)
    const R u_lo = ux - R(0.5), u_hi = ux + R(0.5), m2u = R(-2) * ux;
    inv_line_odd<R>(f[3], f[4], f[5], m110, u_lo, u_hi, m2u);                          // (1, 0)
    inv_line_odd<R>(f[9], f[10], f[11], m101, u_lo, u_hi, m2u);                        // (0, 1)
    inv_line_odd<R>(f[15], f[16], f[17], m121, u_lo, u_hi, m2u);                       // (2, 1)
    inv_line_odd<R>(f[21], f[22], f[23], m112, u_lo, u_hi, m2u);                       // (1, 2)
#pragma unroll
    for (int az = 0; az < 3; ++az)
#pragma unroll
        for (int xi = 0; xi < 3; ++xi)
            inv_line<R>(f[xi + 9 * az], f[xi + 3 + 9 * az], f[xi + 6 + 9 * az], uy, R(tw(xi) * zw(az)));
#pragma unroll
    for (int yi = 0; yi < 3; ++yi)
#pragma unroll
        for (int xi = 0; xi < 3; ++xi)
            inv_line<R>(f[xi + 3 * yi], f[xi + 3 * yi + 9], f[xi + 3 * yi + 18], uz, R(tw(xi) * tw(yi)));
}

// 1/x: for FP32 the hardware estimate refined by one Newton-Raphson step
// r <- r + r (1 - x r) (the error of the estimate is squared, so the result
// is within an ulp or so of the rounded quotient); the FP64 path divides.
template <class R> __device__ __forceinline__ R recip(R x);
template <> __device__ __forceinline__ double recip<double>(double x) { return 1.0 / x; }
template <> __device__ __forceinline__ float recip<float>(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

template <class R>
struct Rates {
    R w1, w2, w3;
    int galilean;
    int param4;
    R p4[6];
};

template <class R>
__device__ __forceinline__ Rates<R> rates_of(const StepArgs &a)
{
    Rates<R> r{pick<R>(a.w1, a.w1f), pick<R>(a.w2, a.w2f), pick<R>(a.w3, a.w3f), a.galilean, a.param4, {}};
#pragma unroll
    for (int k = 0; k < 6; ++k) r.p4[k] = pick<R>(a.p4[k], a.p4f[k]);
    return r;
}

// Rate w raised towards 1 where the cumulant combination X is large against
// the limiter lambda (fourth-order parametrisation): w + (1 - w)|X|/(|X| + lambda).
template <class R>
__device__ __forceinline__ R limited_rate(R w, R X, R lambda)
{
    const R ax = X < R(0) ? -X : X;
    return w + (R(1) - w) * ax / (ax + lambda);
}

// Cumulant collision of one cell, in place on the shifted populations f[27].
// Returns the pre-collision density deviation and velocity.
// PLAIN: every cumulant of order >= 3 relaxes to zero (omega_higher = 1).
template <class R, bool PLAIN>
__device__ __forceinline__ void collide(R *f, const Rates<R> &rt, R &drho_out, R &ux, R &uy, R &uz)
{
    R *m = f;
    const R third = R(1.0 / 3.0), ninth = R(1.0 / 9.0), t27 = R(1.0 / 27.0);
    R drho, rho, ir, d200, d020, d002, k110, k101, k011;
    if (PLAIN) {
        // Only density, momentum and the six second moments enter the
        // relaxation when every higher cumulant is reset: take them as raw
        // moments of the shifted populations by partial sums over x, y, z.
        // (The weights carry no momentum and no off-diagonal second moment;
        // their diagonal second moment 1/3 is the rest offset.)
        R A0[9], A1[9], A2[9];   // per (y, z) line: sum f, sum cx f, sum cx^2 f
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            A2[l] = f[3 * l + 2] + f[3 * l];
            A0[l] = A2[l] + f[3 * l + 1];
            A1[l] = f[3 * l + 2] - f[3 * l];
        }
        R B00[3], B01[3], B02[3], B10[3], B11[3], B20[3];   // per z plane
#pragma unroll
        for (int zi = 0; zi < 3; ++zi) {
            const int lm = 3 * zi, l0 = 3 * zi + 1, lp = 3 * zi + 2;
            B02[zi] = A0[lp] + A0[lm];
            B00[zi] = B02[zi] + A0[l0];
            B01[zi] = A0[lp] - A0[lm];
            B10[zi] = A1[lm] + A1[l0] + A1[lp];
            B11[zi] = A1[lp] - A1[lm];
            B20[zi] = A2[lm] + A2[l0] + A2[lp];
        }
        const R M002 = B00[2] + B00[0];
        const R M000 = M002 + B00[1];
        const R M001 = B00[2] - B00[0];
        const R M010 = B01[0] + B01[1] + B01[2];
        const R M011 = B01[2] - B01[0];
        const R M020 = B02[0] + B02[1] + B02[2];
        const R M100 = B10[0] + B10[1] + B10[2];
        const R M101 = B10[2] - B10[0];
        const R M110 = B11[0] + B11[1] + B11[2];
        const R M200 = B20[0] + B20[1] + B20[2];
        drho = M000;
        rho = R(1) + drho;
        ir = recip<R>(rho);
        ux = M100 * ir;
        uy = M010 * ir;
        uz = M001 * ir;
        // central second moments minus their rest values: kappa_ab - delta_ab/3
        d200 = ((M200 - M100 * ux) - drho * third) * ir;
        d020 = ((M020 - M010 * uy) - drho * third) * ir;
        d002 = ((M002 - M001 * uz) - drho * third) * ir;
        k110 = (M110 - M100 * uy) * ir;
        k101 = (M101 - M100 * uz) * ir;
        k011 = (M011 - M010 * uz) * ir;
    } else {
        // macroscopic quantities (the weights carry no mass flux)
        R jx = R(0), jy = R(0), jz = R(0);
        drho = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            drho += f[i];
            if (cx_of(i) == 1) jx += f[i];
            if (cx_of(i) == -1) jx -= f[i];
            if (cy_of(i) == 1) jy += f[i];
            if (cy_of(i) == -1) jy -= f[i];
            if (cz_of(i) == 1) jz += f[i];
            if (cz_of(i) == -1) jz -= f[i];
        }
        rho = R(1) + drho;
        ir = R(1) / rho;
        ux = jx * ir;
        uy = jy * ir;
        uz = jz * ir;
        chimera_forward<R>(f, ux, uy, uz);
        // second order: normalised deviations from the rest values (1/3 on the diagonal)
        d200 = (m[MI(2, 0, 0)] - drho * third) * ir;
        d020 = (m[MI(0, 2, 0)] - drho * third) * ir;
        d002 = (m[MI(0, 0, 2)] - drho * third) * ir;
        k110 = m[MI(1, 1, 0)] * ir;
        k101 = m[MI(1, 0, 1)] * ir;
        k011 = m[MI(0, 1, 1)] * ir;
    }
    drho_out = drho;

    // relaxation of second order (shear rate on deviators and off-diagonals,
    // bulk rate on the trace), with the Galilean correction built from the
    // velocity-derivative estimates implied by the non-equilibrium moments
    const R w1 = rt.w1, w2 = rt.w2;
    const R Dxy = d200 - d020, Dxz = d200 - d002, dTr = d200 + d020 + d002;
    const R dxu = -R(0.5) * w1 * (R(2) * d200 - d020 - d002) - R(0.5) * w2 * dTr;
    const R dyv = dxu + R(1.5) * w1 * Dxy;
    const R dzw = dxu + R(1.5) * w1 * Dxz;
    const R g = rt.galilean ? R(1) : R(0);
    const R ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const R Dxy_s = (R(1) - w1) * Dxy - g * R(3) * (R(1) - R(0.5) * w1) * (ux2 * dxu - uy2 * dyv);
    const R Dxz_s = (R(1) - w1) * Dxz - g * R(3) * (R(1) - R(0.5) * w1) * (ux2 * dxu - uz2 * dzw);
    const R dTr_s = (R(1) - w2) * dTr - g * R(3) * (R(1) - R(0.5) * w2) * (ux2 * dxu + uy2 * dyv + uz2 * dzw);
    const R s200 = (Dxy_s + Dxz_s + dTr_s) * third;
    const R s020 = s200 - Dxy_s;
    const R s002 = s200 - Dxz_s;
    const R s110 = (R(1) - w1) * k110, s101 = (R(1) - w1) * k101, s011 = (R(1) - w1) * k011;

    // post-collision central moments of orders 3..6 (normalised)
    R s111, s210, s201, s120, s021, s102, s012;   // third
    R s211, s121, s112, e220s, e202s, e022s;      // fourth (e = deviation from 1/9)
    R s122, s212, s221, e222s;                    // fifth, sixth (e = deviation from 1/27)
    if (PLAIN) {
        s111 = s210 = s201 = s120 = s021 = s102 = s012 = R(0);
        s211 = (third + s200) * s011 + R(2) * s110 * s101;
        s121 = (third + s020) * s101 + R(2) * s110 * s011;
        s112 = (third + s002) * s110 + R(2) * s101 * s011;
        e220s = (s200 + s020) * third + s200 * s020 + R(2) * s110 * s110;
        e202s = (s200 + s002) * third + s200 * s002 + R(2) * s101 * s101;
        e022s = (s020 + s002) * third + s020 * s002 + R(2) * s011 * s011;
        s122 = s212 = s221 = R(0);
        e222s = R(0);
    } else {
        const R w3 = rt.w3, r3 = R(1) - w3;
        // third order: cumulants equal central moments
        const R k111 = m[MI(1, 1, 1)] * ir;
        const R k210 = m[MI(2, 1, 0)] * ir, k201 = m[MI(2, 0, 1)] * ir, k120 = m[MI(1, 2, 0)] * ir;
        const R k021 = m[MI(0, 2, 1)] * ir, k102 = m[MI(1, 0, 2)] * ir, k012 = m[MI(0, 1, 2)] * ir;
        // fourth
        const R k211 = m[MI(2, 1, 1)] * ir, k121 = m[MI(1, 2, 1)] * ir, k112 = m[MI(1, 1, 2)] * ir;
        const R e220 = (m[MI(2, 2, 0)] - drho * ninth) * ir;
        const R e202 = (m[MI(2, 0, 2)] - drho * ninth) * ir;
        const R e022 = (m[MI(0, 2, 2)] - drho * ninth) * ir;
        // fifth, sixth
        const R k122 = m[MI(1, 2, 2)] * ir, k212 = m[MI(2, 1, 2)] * ir, k221 = m[MI(2, 2, 1)] * ir;
        const R e222 = (m[MI(2, 2, 2)] - drho * t27) * ir;

        // cumulants of order 4..6 (zero-mean moment->cumulant relations, written
        // on deviations so that the constant parts cancel exactly)
        const R C211 = k211 - ((third + d200) * k011 + R(2) * k110 * k101);
        const R C121 = k121 - ((third + d020) * k101 + R(2) * k110 * k011);
        const R C112 = k112 - ((third + d002) * k110 + R(2) * k101 * k011);
        const R C220 = e220 - ((d200 + d020) * third + d200 * d020 + R(2) * k110 * k110);
        const R C202 = e202 - ((d200 + d002) * third + d200 * d002 + R(2) * k101 * k101);
        const R C022 = e022 - ((d020 + d002) * third + d020 * d002 + R(2) * k011 * k011);
        const R C122 = k122 - ((third + d002) * k120 + (third + d020) * k102 + R(4) * k011 * k111
                               + R(2) * (k101 * k021 + k110 * k012));
        const R C212 = k212 - ((third + d200) * k012 + (third + d002) * k210 + R(4) * k101 * k111
                               + R(2) * (k110 * k102 + k011 * k201));
        const R C221 = k221 - ((third + d200) * k021 + (third + d020) * k201 + R(4) * k110 * k111
                               + R(2) * (k101 * k120 + k011 * k210));
        const R S42 = (d200 + d020 + d002) * ninth + (e022 + e202 + e220) * third
                    + d200 * e022 + d020 * e202 + d002 * e220
                    + R(4) * (k011 * k211 + k101 * k121 + k110 * k112);
        const R S33 = R(4) * k111 * k111 + R(2) * (k120 * k102 + k210 * k012 + k201 * k021);
        const R S222 = R(8) * k110 * k101 * k011
                     + R(2) * (k101 * k101 * (third + d020) + k011 * k011 * (third + d200)
                               + k110 * k110 * (third + d002))
                     + (d200 + d020 + d002) * ninth + (d200 * d020 + d200 * d002 + d020 * d002) * third
                     + d200 * d020 * d002;
        const R C222 = e222 - S42 - S33 + R(2) * S222;

        // post-collision cumulants of orders 3..6: one rate omega_higher for
        // all of them, or the fourth-order parametrisation
        R c111, c210, c201, c120, c021, c102, c012, c211, c121, c112, c220, c202, c022, c122, c212, c221, c222;
        if (rt.param4) {
            // third order in the combinations of Geier et al. 2017: sums with
            // omega3, differences with omega4, C_111 with omega5, each limited
            const R lam = rt.p4[5];
            const R p1 = k210 + k012, m1 = k210 - k012;
            const R p2 = k201 + k021, m2 = k201 - k021;
            const R p3 = k120 + k102, m3 = k120 - k102;
            const R p1s = (R(1) - limited_rate<R>(rt.p4[0], p1, lam)) * p1;
            const R m1s = (R(1) - limited_rate<R>(rt.p4[1], m1, lam)) * m1;
            const R p2s = (R(1) - limited_rate<R>(rt.p4[0], p2, lam)) * p2;
            const R m2s = (R(1) - limited_rate<R>(rt.p4[1], m2, lam)) * m2;
            const R p3s = (R(1) - limited_rate<R>(rt.p4[0], p3, lam)) * p3;
            const R m3s = (R(1) - limited_rate<R>(rt.p4[1], m3, lam)) * m3;
            c210 = R(0.5) * (p1s + m1s); c012 = R(0.5) * (p1s - m1s);
            c201 = R(0.5) * (p2s + m2s); c021 = R(0.5) * (p2s - m2s);
            c120 = R(0.5) * (p3s + m3s); c102 = R(0.5) * (p3s - m3s);
            c111 = (R(1) - limited_rate<R>(rt.p4[2], k111, lam)) * k111;
            // fourth order: the equilibria carrying the velocity gradients
            c220 = rt.p4[3] * (dxu + dyv);
            c202 = rt.p4[3] * (dxu + dzw);
            c022 = rt.p4[3] * (dyv + dzw);
            c211 = rt.p4[4] * k011;
            c121 = rt.p4[4] * k101;
            c112 = rt.p4[4] * k110;
            c122 = c212 = c221 = c222 = R(0);
        } else {
            c111 = r3 * k111;
            c210 = r3 * k210; c201 = r3 * k201; c120 = r3 * k120;
            c021 = r3 * k021; c102 = r3 * k102; c012 = r3 * k012;
            c211 = r3 * C211; c121 = r3 * C121; c112 = r3 * C112;
            c220 = r3 * C220; c202 = r3 * C202; c022 = r3 * C022;
            c122 = r3 * C122; c212 = r3 * C212; c221 = r3 * C221;
            c222 = r3 * C222;
        }
        // rebuild central moments order by order from the post-collision
        // lower orders
        s111 = c111;
        s210 = c210; s201 = c201; s120 = c120;
        s021 = c021; s102 = c102; s012 = c012;
        s211 = c211 + (third + s200) * s011 + R(2) * s110 * s101;
        s121 = c121 + (third + s020) * s101 + R(2) * s110 * s011;
        s112 = c112 + (third + s002) * s110 + R(2) * s101 * s011;
        e220s = c220 + (s200 + s020) * third + s200 * s020 + R(2) * s110 * s110;
        e202s = c202 + (s200 + s002) * third + s200 * s002 + R(2) * s101 * s101;
        e022s = c022 + (s020 + s002) * third + s020 * s002 + R(2) * s011 * s011;
        s122 = c122 + (third + s002) * s120 + (third + s020) * s102 + R(4) * s011 * s111
             + R(2) * (s101 * s021 + s110 * s012);
        s212 = c212 + (third + s200) * s012 + (third + s002) * s210 + R(4) * s101 * s111
             + R(2) * (s110 * s102 + s011 * s201);
        s221 = c221 + (third + s200) * s021 + (third + s020) * s201 + R(4) * s110 * s111
             + R(2) * (s101 * s120 + s011 * s210);
        e222s = c222;   // plus the product terms added below
    }
    {
        // sixth order: add sum(4,2) + sum(3,3) - 2 sum(2,2,2) of post-collision moments
        const R S42s = (s200 + s020 + s002) * ninth + (e022s + e202s + e220s) * third
                     + s200 * e022s + s020 * e202s + s002 * e220s
                     + R(4) * (s011 * s211 + s101 * s121 + s110 * s112);
        const R S33s = R(4) * s111 * s111 + R(2) * (s120 * s102 + s210 * s012 + s201 * s021);
        const R S222s = R(8) * s110 * s101 * s011
                      + R(2) * (s101 * s101 * (third + s020) + s011 * s011 * (third + s200)
                                + s110 * s110 * (third + s002))
                      + (s200 + s020 + s002) * ninth + (s200 * s020 + s200 * s002 + s020 * s002) * third
                      + s200 * s020 * s002;
        e222s += S42s + S33s - R(2) * S222s;
    }

    if (PLAIN) {
        // odd orders are zero: only the even-order moments enter the inverse
        chimera_inverse_even<R>(f, ux, uy, uz, drho, rho * s200 + drho * third, rho * s020 + drho * third,
                                rho * s002 + drho * third, rho * s110, rho * s101, rho * s011, rho * s211,
                                rho * s121, rho * s112, rho * e220s + drho * ninth, rho * e202s + drho * ninth,
                                rho * e022s + drho * ninth, rho * e222s + drho * t27);
        return;
    }

    // back to non-normalised central moment deviations
    m[MI(0, 0, 0)] = drho;
    m[MI(1, 0, 0)] = R(0); m[MI(0, 1, 0)] = R(0); m[MI(0, 0, 1)] = R(0);
    m[MI(2, 0, 0)] = rho * s200 + drho * third;
    m[MI(0, 2, 0)] = rho * s020 + drho * third;
    m[MI(0, 0, 2)] = rho * s002 + drho * third;
    m[MI(1, 1, 0)] = rho * s110; m[MI(1, 0, 1)] = rho * s101; m[MI(0, 1, 1)] = rho * s011;
    m[MI(1, 1, 1)] = rho * s111;
    m[MI(2, 1, 0)] = rho * s210; m[MI(2, 0, 1)] = rho * s201; m[MI(1, 2, 0)] = rho * s120;
    m[MI(0, 2, 1)] = rho * s021; m[MI(1, 0, 2)] = rho * s102; m[MI(0, 1, 2)] = rho * s012;
    m[MI(2, 1, 1)] = rho * s211; m[MI(1, 2, 1)] = rho * s121; m[MI(1, 1, 2)] = rho * s112;
    m[MI(2, 2, 0)] = rho * e220s + drho * ninth;
    m[MI(2, 0, 2)] = rho * e202s + drho * ninth;
    m[MI(0, 2, 2)] = rho * e022s + drho * ninth;
    m[MI(1, 2, 2)] = rho * s122; m[MI(2, 1, 2)] = rho * s212; m[MI(2, 2, 1)] = rho * s221;
    m[MI(2, 2, 2)] = rho * e222s + drho * t27;

    chimera_inverse<R>(f, ux, uy, uz);
}

#undef MI

// Latch instability: density outside (0.5, 1.5) or not a number.
template <class R>
__device__ __forceinline__ void check_density(R drho, int *status)
{
    if (!(drho > R(-0.5) && drho < R(0.5))) atomicOr(status, STATUS_UNSTABLE);
}

}  // namespace lbm
