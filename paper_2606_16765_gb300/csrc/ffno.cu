// ffno.cu -- the factorised Fourier Neural Operator of include/ffno.h:
// forward, hand-written backward and Adam in FP32 (activations and
// arithmetic), one thread per output element.
//
// Fields are [batch][channel][z][y][x].  A spectrum along axis d keeps the
// field's layout with that axis's samples replaced by its first m_d wave
// numbers (complex, float2), so the three axes share one indexing rule:
// extents (ez, ey, ex) with e_d = m_d, element (b, c, iz, iy, ix).
//   k_dft       V(k) = w_k sum_n v(n) exp(-2 pi i k n / L)      (w_k = 1, or
//               c_k / L for the adjoint of the inverse)
//   k_idft      u(n) [+]= Re sum_k a_k G(k) exp(+2 pi i k n / L)  (a_k = c_k / L
//               for the inverse, 1 for the adjoint of the forward)
//   k_mix       W(b, o, ., k) = sum_i V(b, i, ., k) R(i, o, k), or its adjoint
//               gV(b, i, ., k) = sum_o gW(b, o, ., k) conj R(i, o, k)
//   k_gradR     gR(i, o, k) = sum_{b, .} gW(b, o, ., k) conj V(b, i, ., k)
//   k_pw        y = act(W x + b) [+ residual], pre-activation kept
//   k_act_bwd   g * act'(kept)
//   k_pw_in     gx [+]= W^T g
//   k_outer     gW = sum_{b, n} g x^T, gb = sum g (fixed order, no atomics)
//   k_mse_*     masked mean square error (FP64 block partials) and its gradient
//   k_adam      Adam on the flat FP32 parameters (real and imaginary parts
//               as separate entries)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ffno.h"
#include "sm_count.h"

namespace {

constexpr int TPB = 256;
enum { ACT_NONE = 0, ACT_GELU = 1, ACT_SIREN = 2 };

int grid_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + TPB - 1) / TPB, (int64_t)gb300::sm_count() * 16));
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Extents of a field or spectrum: (e[0], e[1], e[2]) = (z, y, x) extents.
struct Ext {
    int e[3];
    __host__ __device__ int64_t n() const { return (int64_t)e[0] * e[1] * e[2]; }
};

__device__ __forceinline__ void unflat(int64_t r, const Ext &x, int &iz, int &iy, int &ix)
{
    ix = (int)(r % x.e[2]);
    const int64_t q = r / x.e[2];
    iy = (int)(q % x.e[1]);
    iz = (int)(q / x.e[1]);
}

__device__ __forceinline__ int64_t flat(const Ext &x, int iz, int iy, int ix)
{
    return ((int64_t)iz * x.e[1] + iy) * x.e[2] + ix;
}

// forward transform along axis d: v over extents fe (real), V over se
// (e_d = m); rows = batch x channels; tw [m][L] = (cos, sin)(2 pi k s / L)
__global__ void k_dft(const float *v, float2 *V, int64_t rows, Ext fe, Ext se, int d, const float2 *tw,
                      const float *wk)
{
    const int L = fe.e[d];
    const int64_t ns = se.n(), total = rows * ns;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / ns, r = t % ns;
        int c[3];
        unflat(r, se, c[0], c[1], c[2]);
        const int k = c[d];
        float re = 0.f, im = 0.f;
        for (int s = 0; s < L; ++s) {
            c[d] = s;
            const float x = v[row * fe.n() + flat(fe, c[0], c[1], c[2])];
            const float2 w = tw[(int64_t)k * L + s];
            re += x * w.x;                              // x exp(-i theta)
            im -= x * w.y;
        }
        const float a = wk ? wk[k] : 1.f;
        V[t] = make_float2(re * a, im * a);
    }
}

// inverse transform along axis d: G over se (e_d = m) to u over fe (real)
__global__ void k_idft(const float2 *G, float *u, int64_t rows, Ext fe, Ext se, int d, const float2 *tw,
                       const float *ak, int accumulate)
{
    const int L = fe.e[d], m = se.e[d];
    const int64_t nf = fe.n(), total = rows * nf;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = t / nf, r = t % nf;
        int c[3];
        unflat(r, fe, c[0], c[1], c[2]);
        const int s = c[d];
        float acc = 0.f;
        for (int k = 0; k < m; ++k) {
            c[d] = k;
            const float2 g = G[row * se.n() + flat(se, c[0], c[1], c[2])];
            const float2 w = tw[(int64_t)k * L + s];
            acc += ak[k] * (g.x * w.x - g.y * w.y);     // Re[g exp(+i theta)]
        }
        u[t] = accumulate ? u[t] + acc : acc;
    }
}

// R (i, o, k) as interleaved floats [i][o][k][re, im] (no alignment assumed)
__device__ __forceinline__ float2 rw(const float *R, int C, int m, int i, int o, int k)
{
    const int64_t j = (((int64_t)i * C + o) * m + k) * 2;
    return make_float2(R[j], R[j + 1]);
}

// channel mixing of a spectrum along axis d (C channels, batch B)
__global__ void k_mix(const float2 *V, const float *R, float2 *Wout, int B, int C, Ext se, int d, int adj)
{
    const int m = se.e[d];
    const int64_t ns = se.n(), total = (int64_t)B * C * ns;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t % ns, bc = t / ns;
        const int c = (int)(bc % C);
        const int64_t b = bc / C;
        int e[3];
        unflat(r, se, e[0], e[1], e[2]);
        const int k = e[d];
        float re = 0.f, im = 0.f;
        for (int q = 0; q < C; ++q) {
            const float2 a = V[(b * C + q) * ns + r];
            if (!adj) {                                     // out c = o, in q = i: a R(q, c, k)
                const float2 w = rw(R, C, m, q, c, k);
                re += a.x * w.x - a.y * w.y;
                im += a.x * w.y + a.y * w.x;
            } else {                                        // out c = i, in q = o: a conj R(c, q, k)
                const float2 w = rw(R, C, m, c, q, k);
                re += a.x * w.x + a.y * w.y;
                im += a.y * w.x - a.x * w.y;
            }
        }
        Wout[t] = make_float2(re, im);
    }
}

// gR(i, o, k) = sum over batch and the other positions of gW(b, o, ., k) conj V(b, i, ., k)
__global__ void k_gradR(const float2 *gW, const float2 *V, float *gR, int B, int C, Ext se, int d)
{
    const int m = se.e[d];
    const int64_t ns = se.n();
    Ext o2 = se;
    o2.e[d] = 1;                                            // the positions with k fixed
    const int64_t np = o2.n(), total = (int64_t)C * C * m;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % m);
        const int o = (int)((t / m) % C);
        const int i = (int)(t / ((int64_t)m * C));
        float re = 0.f, im = 0.f;
        for (int b = 0; b < B; ++b)
            for (int64_t p = 0; p < np; ++p) {
                int e[3];
                unflat(p, o2, e[0], e[1], e[2]);
                e[d] = k;
                const int64_t r = flat(se, e[0], e[1], e[2]);
                const float2 g = gW[((int64_t)b * C + o) * ns + r], v = V[((int64_t)b * C + i) * ns + r];
                re += g.x * v.x + g.y * v.y;                // g conj(v)
                im += g.y * v.x - g.x * v.y;
            }
        gR[2 * t] = re;
        gR[2 * t + 1] = im;
    }
}

// y(b, o, n) = act(sum_i W(o, i) x(b, i, n) + b(o)) [+ res(b, o, n)]; keep = the
// pre-activation (GELU) or cos(omega0 z) (SIREN)
__global__ void k_pw(const float *x, int ci, int co, const float *W, const float *bias, const float *res, float *keep,
                     float *y, int act, float w0, int B, int64_t N)
{
    const int64_t total = (int64_t)B * co * N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = t % N, bo = t / N;
        const int o = (int)(bo % co);
        const int64_t b = bo / co;
        float z = bias[o];
        for (int i = 0; i < ci; ++i) z += W[(int64_t)o * ci + i] * x[(b * ci + i) * N + n];
        float out = z;
        if (act == ACT_GELU) {
            if (keep) keep[t] = z;
            out = gelu(z);
        } else if (act == ACT_SIREN) {
            float sn, cs;
            sincosf(w0 * z, &sn, &cs);
            if (keep) keep[t] = cs;
            out = sn;
        }
        y[t] = res ? res[t] + out : out;
    }
}

// g *= act'(kept), in place
__global__ void k_act_bwd(float *g, const float *kept, int act, float w0, int64_t n)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        g[t] *= act == ACT_GELU ? gelu_grad(kept[t]) : w0 * kept[t];
}

// gx(b, i, n) [+]= sum_o W(o, i) g(b, o, n)
__global__ void k_pw_in(const float *g, int co, int ci, const float *W, float *gx, int B, int64_t N, int accumulate)
{
    const int64_t total = (int64_t)B * ci * N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = t % N, bi = t / N;
        const int i = (int)(bi % ci);
        const int64_t b = bi / ci;
        float s = 0.f;
        for (int o = 0; o < co; ++o) s += W[(int64_t)o * ci + i] * g[(b * co + o) * N + n];
        gx[t] = accumulate ? gx[t] + s : s;
    }
}

// gW(o, i) = sum_{b, n} g(b, o, n) x(b, i, n); gb(o) = sum g(b, o, n).  One
// block per (o, i) (i = ci: the bias), a fixed-order block reduction.
__global__ void __launch_bounds__(TPB) k_outer(const float *g, int co, const float *x, int ci, float *gW, float *gb,
                                               int B, int64_t N)
{
    __shared__ float sh[TPB];
    const int o = (int)(blockIdx.x / (ci + 1)), i = (int)(blockIdx.x % (ci + 1));
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
            const float gv = g[((int64_t)b * co + o) * N + n];
            s += i < ci ? gv * x[((int64_t)b * ci + i) * N + n] : gv;
        }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = TPB / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (i < ci) gW[(int64_t)o * ci + i] = sh[0];
        else gb[o] = sh[0];
    }
}

// masked mean square error: per-block FP64 partials of sum m (y - t)^2 and
// sum m, then their fixed-order sum
__global__ void __launch_bounds__(TPB) k_mse_partial(const float *y, const float *tt, const float *msk, int C, int B,
                                                     int64_t N, double *part)
{
    __shared__ double s1[TPB], s2[TPB];
    double a = 0.0, w = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)B * N;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / N, n = t % N;
        const double mm = msk[t];
        w += mm;
        for (int c = 0; c < C; ++c) {
            const double d = (double)y[(b * C + c) * N + n] - tt[(b * C + c) * N + n];
            a += mm * d * d;
        }
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = w;
    __syncthreads();
    for (int h = TPB / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            s1[threadIdx.x] += s1[threadIdx.x + h];
            s2[threadIdx.x] += s2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

__global__ void k_mse_final(const double *part, int nb, int C, double *res)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, w = 0.0;
        for (int k = 0; k < nb; ++k) {
            a += part[2 * k];
            w += part[2 * k + 1];
        }
        res[0] = a / (C * w);        // loss
        res[1] = w;                  // sum of the weights
    }
}

// dL/dy = 2 m (y - t) / (C sum m)
__global__ void k_mse_grad(const float *y, const float *tt, const float *msk, int C, int B, int64_t N,
                           const double *res, float *gy)
{
    const int64_t total = (int64_t)B * C * N;
    const double sc = 2.0 / (C * res[1]);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = t % N, b = t / ((int64_t)C * N);
        gy[t] = (float)(sc * msk[b * N + n] * ((double)y[t] - tt[t]));
    }
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float a = b1 * m1[k] + (1.f - b1) * gk;
        const float v = b2 * m2[k] + (1.f - b2) * gk * gk;
        m1[k] = a;
        m2[k] = v;
        p[k] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// context and C ABI
// ---------------------------------------------------------------------------
struct ffno_ctx {
    ffno_config c{};
    cudaStream_t s = nullptr;
    std::string err;
    int64_t N = 0, np = 0, adam_t = 0;
    Ext fe{}, se[3]{};
    int64_t oP1w = 0, oP1b = 0, oP2w = 0, oP2b = 0, oQ1w = 0, oQ1b = 0, oQ2w = 0, oQ2b = 0;
    std::vector<int64_t> oR, oF1w, oF1b, oF2w, oF2b;        // oR[3 l + d]
    std::vector<void *> allocs;
    float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
    float2 *tw[3] = {nullptr, nullptr, nullptr};
    float *ck[3] = {nullptr, nullptr, nullptr}, *ones[3] = {nullptr, nullptr, nullptr};
    float *xin = nullptr, *tin = nullptr, *min = nullptr, *apre = nullptr, *a = nullptr, *hkeep = nullptr, *h = nullptr,
          *y = nullptr;
    std::vector<float *> v, u, z, hff;
    std::vector<float2 *> spec;                              // spec[3 l + d]
    float2 *mixw = nullptr, *mixw2 = nullptr;
    float *gy = nullptr, *gh = nullptr, *gv = nullptr, *gz = nullptr, *gu = nullptr, *ga = nullptr;
    double *part = nullptr, *res = nullptr;
    int nb_loss = 0;
};

namespace {

std::string g_ffno_err;

lbm_status ffail(ffno_ctx *f, lbm_status st, const std::string &m)
{
    if (f) f->err = m;
    else g_ffno_err = m;
    return st;
}

#define FCK(x)                                                                                         \
    do {                                                                                               \
        cudaError_t e_ = (x);                                                                          \
        if (e_ != cudaSuccess) return ffail(f, LBM_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
lbm_status alloc(ffno_ctx *f, T *&p, int64_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ffail(f, LBM_ERR_OOM, "device allocation of " + std::to_string(count * (int64_t)sizeof(T)) + " bytes failed");
    }
    f->allocs.push_back(q);
    p = static_cast<T *>(q);
    return LBM_OK;
}

uint64_t splitmix(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double unif(uint64_t &s) { return 2.0 * ((splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0; }

bool is_host(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged;
}

std::string validate(const ffno_config &c)
{
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) return "grid extents must be positive";
    if (c.cin < 1 || c.width < 1 || c.cout < 1 || c.layers < 0 || c.ff_hidden < 1 || c.hidden < 1 || c.lift_hidden < 1)
        return "channel counts must be positive";
    if (c.mx < 1 || c.my < 1 || c.mz < 1 || c.mx > c.nx / 2 + 1 || c.my > c.ny / 2 + 1 || c.mz > c.nz / 2 + 1)
        return "wave numbers per axis must lie in [1, L/2 + 1]";
    if (c.max_batch < 1) return "max_batch must be positive";
    if (!(c.omega0 > 0.f)) return "omega0 must be positive";
    return "";
}

}  // namespace

extern "C" void ffno_config_default(ffno_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->nx = 128; c->ny = 64; c->nz = 64;
    c->cin = 4; c->width = 32; c->cout = 4;
    c->mx = 32; c->my = 16; c->mz = 16;
    c->layers = 4; c->ff_hidden = 32; c->hidden = 128; c->lift_hidden = 32;
    c->max_batch = 8; c->omega0 = 30.f; c->seed = 0;
}

extern "C" lbm_status ffno_destroy(ffno_ctx *f)
{
    if (!f) return LBM_ERR_ARG;
    for (void *p : f->allocs) cudaFree(p);
    delete f;
    return LBM_OK;
}

extern "C" int64_t ffno_num_params(const ffno_ctx *f) { return f ? f->np : -1; }
extern "C" const char *ffno_last_error(const ffno_ctx *f) { return f ? f->err.c_str() : g_ffno_err.c_str(); }

extern "C" lbm_status ffno_create(const ffno_config *cfg, void *stream, ffno_ctx **out)
{
    if (!cfg || !out) return ffail(nullptr, LBM_ERR_ARG, "null argument");
    *out = nullptr;
    const std::string bad = validate(*cfg);
    if (!bad.empty()) return ffail(nullptr, LBM_ERR_ARG, bad);
    ffno_ctx *f = new ffno_ctx();
    f->c = *cfg;
    f->s = static_cast<cudaStream_t>(stream);
    const ffno_config &c = f->c;
    const int W = c.width, H = c.ff_hidden, LH = c.lift_hidden, L = c.layers, B = c.max_batch;
    f->N = (int64_t)c.nx * c.ny * c.nz;
    f->fe = Ext{{c.nz, c.ny, c.nx}};
    const int m[3] = {c.mz, c.my, c.mx};
    for (int d = 0; d < 3; ++d) {
        f->se[d] = f->fe;
        f->se[d].e[d] = m[d];
    }
    // flat parameter layout (include/ffno.h)
    int64_t o = 0;
    auto take = [&](int64_t n) { const int64_t r = o; o += n; return r; };
    f->oP1w = take((int64_t)LH * c.cin); f->oP1b = take(LH);
    f->oP2w = take((int64_t)W * LH); f->oP2b = take(W);
    for (int l = 0; l < L; ++l) {
        for (int d = 0; d < 3; ++d) f->oR.push_back(take((int64_t)W * W * m[d] * 2));
        f->oF1w.push_back(take((int64_t)H * W)); f->oF1b.push_back(take(H));
        f->oF2w.push_back(take((int64_t)W * H)); f->oF2b.push_back(take(W));
    }
    f->oQ1w = take((int64_t)c.hidden * W); f->oQ1b = take(c.hidden);
    f->oQ2w = take((int64_t)c.cout * c.hidden); f->oQ2b = take(c.cout);
    f->np = o;
    lbm_status st = LBM_OK;
    auto A = [&](auto *&p, int64_t n) { if (st == LBM_OK) st = alloc(f, p, n); };
    A(f->params, f->np); A(f->grads, f->np); A(f->m1, f->np); A(f->m2, f->np);
    const int64_t BN = (int64_t)B * f->N;
    A(f->xin, BN * c.cin); A(f->tin, BN * c.cout); A(f->min, BN);
    A(f->apre, BN * LH); A(f->a, BN * LH); A(f->hkeep, BN * c.hidden); A(f->h, BN * c.hidden); A(f->y, BN * c.cout);
    f->v.assign(L + 1, nullptr); f->u.assign(L, nullptr); f->z.assign(L, nullptr); f->hff.assign(L, nullptr);
    f->spec.assign(3 * L, nullptr);
    for (int l = 0; l <= L; ++l) A(f->v[l], BN * W);
    int64_t smax = 0;
    for (int d = 0; d < 3; ++d) smax = std::max(smax, f->se[d].n());
    for (int l = 0; l < L; ++l) {
        A(f->u[l], BN * W); A(f->z[l], BN * H); A(f->hff[l], BN * H);
        for (int d = 0; d < 3; ++d) A(f->spec[3 * l + d], (int64_t)B * W * f->se[d].n());
    }
    A(f->mixw, (int64_t)B * W * smax); A(f->mixw2, (int64_t)B * W * smax);
    const int64_t cmax = std::max<int64_t>({(int64_t)W, (int64_t)H, (int64_t)LH, (int64_t)c.hidden, (int64_t)c.cout});
    A(f->gy, BN * c.cout); A(f->gh, BN * c.hidden); A(f->gv, BN * W); A(f->gz, BN * cmax); A(f->gu, BN * W);
    A(f->ga, BN * LH);
    f->nb_loss = grid_for(BN);
    A(f->part, 2 * (int64_t)f->nb_loss); A(f->res, 2);
    for (int d = 0; d < 3; ++d) { A(f->tw[d], (int64_t)m[d] * f->fe.e[d]); A(f->ck[d], m[d]); A(f->ones[d], m[d]); }
    if (st != LBM_OK) {
        const std::string e = f->err;
        ffno_destroy(f);
        return ffail(nullptr, st, e);
    }
    // twiddle tables and inverse weights (FP64 on the host)
    for (int d = 0; d < 3; ++d) {
        const int Ld = f->fe.e[d];
        std::vector<float2> tw((size_t)m[d] * Ld);
        std::vector<float> ck(m[d]), on(m[d], 1.f);
        for (int k = 0; k < m[d]; ++k) {
            for (int s = 0; s < Ld; ++s) {
                const double ang = 2.0 * M_PI * (double)(((int64_t)k * s) % Ld) / Ld;
                tw[(size_t)k * Ld + s] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            }
            const double cw = (k == 0 || (Ld % 2 == 0 && k == Ld / 2)) ? 1.0 : 2.0;
            ck[k] = (float)(cw / Ld);
        }
        if (cudaMemcpy(f->tw[d], tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(f->ck[d], ck.data(), ck.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(f->ones[d], on.data(), on.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            ffno_destroy(f);
            return ffail(nullptr, LBM_ERR_CUDA, "table upload failed");
        }
    }
    // initial parameters: uniform within 1/sqrt(fan_in), spectral weights
    // within 1/width^2, SIREN within 1/fan_in (first layer) and
    // sqrt(6/fan_in)/omega0 (output layer)
    std::vector<float> p((size_t)f->np);
    uint64_t sd = c.seed * 0x2545F4914F6CDD1Dull + 17;
    auto fill = [&](int64_t off, int64_t n, double sc) { for (int64_t k = 0; k < n; ++k) p[off + k] = (float)(sc * unif(sd)); };
    fill(f->oP1w, (int64_t)LH * c.cin, 1 / std::sqrt((double)c.cin)); fill(f->oP1b, LH, 1 / std::sqrt((double)c.cin));
    fill(f->oP2w, (int64_t)W * LH, 1 / std::sqrt((double)LH)); fill(f->oP2b, W, 1 / std::sqrt((double)LH));
    for (int l = 0; l < L; ++l) {
        for (int d = 0; d < 3; ++d) fill(f->oR[3 * l + d], (int64_t)W * W * m[d] * 2, 1.0 / ((double)W * W));
        fill(f->oF1w[l], (int64_t)H * W, 1 / std::sqrt((double)W)); fill(f->oF1b[l], H, 1 / std::sqrt((double)W));
        fill(f->oF2w[l], (int64_t)W * H, 1 / std::sqrt((double)H)); fill(f->oF2b[l], W, 1 / std::sqrt((double)H));
    }
    fill(f->oQ1w, (int64_t)c.hidden * W, 1.0 / W); fill(f->oQ1b, c.hidden, 1 / std::sqrt((double)W));
    fill(f->oQ2w, (int64_t)c.cout * c.hidden, std::sqrt(6.0 / c.hidden) / c.omega0);
    fill(f->oQ2b, c.cout, 1 / std::sqrt((double)c.hidden));
    if (cudaMemcpy(f->params, p.data(), p.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(f->m1, 0, f->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(f->m2, 0, f->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(f->grads, 0, f->np * sizeof(float)) != cudaSuccess) {
        ffno_destroy(f);
        return ffail(nullptr, LBM_ERR_CUDA, "parameter upload failed");
    }
    *out = f;
    return LBM_OK;
}

extern "C" lbm_status ffno_set_params(ffno_ctx *f, const float *src)
{
    if (!f || !src) return ffail(f, LBM_ERR_ARG, "null argument");
    FCK(cudaMemcpyAsync(f->params, src, f->np * sizeof(float), cudaMemcpyDefault, f->s));
    FCK(cudaStreamSynchronize(f->s));
    f->adam_t = 0;
    FCK(cudaMemsetAsync(f->m1, 0, f->np * sizeof(float), f->s));
    FCK(cudaMemsetAsync(f->m2, 0, f->np * sizeof(float), f->s));
    return LBM_OK;
}

static lbm_status copy_out(ffno_ctx *f, float *dst, const float *src)
{
    if (!f || !dst) return ffail(f, LBM_ERR_ARG, "null argument");
    FCK(cudaMemcpyAsync(dst, src, f->np * sizeof(float), cudaMemcpyDefault, f->s));
    FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

extern "C" lbm_status ffno_get_params(ffno_ctx *f, float *dst) { return copy_out(f, dst, f ? f->params : nullptr); }
extern "C" lbm_status ffno_get_grads(ffno_ctx *f, float *dst) { return copy_out(f, dst, f ? f->grads : nullptr); }

extern "C" lbm_status ffno_sync(ffno_ctx *f)
{
    if (!f) return LBM_ERR_ARG;
    FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

namespace {

// the forward pass of `B` samples staged in f->xin; every activation kept
void forward_impl(ffno_ctx *f, int B)
{
    const ffno_config &c = f->c;
    const int W = c.width, H = c.ff_hidden, LH = c.lift_hidden;
    const int64_t N = f->N, BN = (int64_t)B * N;
    const float *P = f->params;
    cudaStream_t s = f->s;
    k_pw<<<grid_for(BN * LH), TPB, 0, s>>>(f->xin, c.cin, LH, P + f->oP1w, P + f->oP1b, nullptr, f->apre, f->a,
                                           ACT_GELU, c.omega0, B, N);
    k_pw<<<grid_for(BN * W), TPB, 0, s>>>(f->a, LH, W, P + f->oP2w, P + f->oP2b, nullptr, nullptr, f->v[0], ACT_NONE,
                                          c.omega0, B, N);
    for (int l = 0; l < c.layers; ++l) {
        for (int d = 0; d < 3; ++d) {
            const int64_t ns = (int64_t)B * W * f->se[d].n();
            float2 *V = f->spec[3 * l + d];
            k_dft<<<grid_for(ns), TPB, 0, s>>>(f->v[l], V, (int64_t)B * W, f->fe, f->se[d], d, f->tw[d], nullptr);
            k_mix<<<grid_for(ns), TPB, 0, s>>>(V, P + f->oR[3 * l + d], f->mixw, B, W, f->se[d], d, 0);
            k_idft<<<grid_for(BN * W), TPB, 0, s>>>(f->mixw, f->u[l], (int64_t)B * W, f->fe, f->se[d], d, f->tw[d],
                                                    f->ck[d], d > 0);
        }
        k_pw<<<grid_for(BN * H), TPB, 0, s>>>(f->u[l], W, H, P + f->oF1w[l], P + f->oF1b[l], nullptr, f->z[l], f->hff[l],
                                              ACT_GELU, c.omega0, B, N);
        k_pw<<<grid_for(BN * W), TPB, 0, s>>>(f->hff[l], H, W, P + f->oF2w[l], P + f->oF2b[l], f->v[l], nullptr,
                                              f->v[l + 1], ACT_NONE, c.omega0, B, N);
    }
    k_pw<<<grid_for(BN * c.hidden), TPB, 0, s>>>(f->v[c.layers], W, c.hidden, P + f->oQ1w, P + f->oQ1b, nullptr,
                                                 f->hkeep, f->h, ACT_SIREN, c.omega0, B, N);
    k_pw<<<grid_for(BN * c.cout), TPB, 0, s>>>(f->h, c.hidden, c.cout, P + f->oQ2w, P + f->oQ2b, nullptr, nullptr,
                                               f->y, ACT_NONE, c.omega0, B, N);
}

// gradients of the loss whose output gradient is in f->gy
void backward_impl(ffno_ctx *f, int B)
{
    const ffno_config &c = f->c;
    const int W = c.width, H = c.ff_hidden, LH = c.lift_hidden;
    const int64_t N = f->N, BN = (int64_t)B * N;
    const float *P = f->params;
    float *G = f->grads;
    cudaStream_t s = f->s;
    k_outer<<<c.cout * (c.hidden + 1), TPB, 0, s>>>(f->gy, c.cout, f->h, c.hidden, G + f->oQ2w, G + f->oQ2b, B, N);
    k_pw_in<<<grid_for(BN * c.hidden), TPB, 0, s>>>(f->gy, c.cout, c.hidden, P + f->oQ2w, f->gh, B, N, 0);
    k_act_bwd<<<grid_for(BN * c.hidden), TPB, 0, s>>>(f->gh, f->hkeep, ACT_SIREN, c.omega0, BN * c.hidden);
    k_outer<<<c.hidden * (W + 1), TPB, 0, s>>>(f->gh, c.hidden, f->v[c.layers], W, G + f->oQ1w, G + f->oQ1b, B, N);
    k_pw_in<<<grid_for(BN * W), TPB, 0, s>>>(f->gh, c.hidden, W, P + f->oQ1w, f->gv, B, N, 0);
    for (int l = c.layers - 1; l >= 0; --l) {
        // v_{l+1} = v_l + F2 GELU(F1 u + b1) + b2
        k_outer<<<W * (H + 1), TPB, 0, s>>>(f->gv, W, f->hff[l], H, G + f->oF2w[l], G + f->oF2b[l], B, N);
        k_pw_in<<<grid_for(BN * H), TPB, 0, s>>>(f->gv, W, H, P + f->oF2w[l], f->gz, B, N, 0);
        k_act_bwd<<<grid_for(BN * H), TPB, 0, s>>>(f->gz, f->z[l], ACT_GELU, c.omega0, BN * H);
        k_outer<<<H * (W + 1), TPB, 0, s>>>(f->gz, H, f->u[l], W, G + f->oF1w[l], G + f->oF1b[l], B, N);
        k_pw_in<<<grid_for(BN * W), TPB, 0, s>>>(f->gz, H, W, P + f->oF1w[l], f->gu, B, N, 0);
        // the residual path keeps gv; each axis adds the adjoint of its branch
        for (int d = 0; d < 3; ++d) {
            const int64_t ns = (int64_t)B * W * f->se[d].n();
            const int m = f->se[d].e[d];
            k_dft<<<grid_for(ns), TPB, 0, s>>>(f->gu, f->mixw, (int64_t)B * W, f->fe, f->se[d], d, f->tw[d], f->ck[d]);
            k_gradR<<<grid_for((int64_t)W * W * m), TPB, 0, s>>>(f->mixw, f->spec[3 * l + d], G + f->oR[3 * l + d], B, W,
                                                                 f->se[d], d);
            k_mix<<<grid_for(ns), TPB, 0, s>>>(f->mixw, P + f->oR[3 * l + d], f->mixw2, B, W, f->se[d], d, 1);
            k_idft<<<grid_for(BN * W), TPB, 0, s>>>(f->mixw2, f->gv, (int64_t)B * W, f->fe, f->se[d], d, f->tw[d],
                                                    f->ones[d], 1);
        }
    }
    k_outer<<<W * (LH + 1), TPB, 0, s>>>(f->gv, W, f->a, LH, G + f->oP2w, G + f->oP2b, B, N);
    k_pw_in<<<grid_for(BN * LH), TPB, 0, s>>>(f->gv, W, LH, P + f->oP2w, f->ga, B, N, 0);
    k_act_bwd<<<grid_for(BN * LH), TPB, 0, s>>>(f->ga, f->apre, ACT_GELU, c.omega0, BN * LH);
    k_outer<<<LH * (c.cin + 1), TPB, 0, s>>>(f->ga, LH, f->xin, c.cin, G + f->oP1w, G + f->oP1b, B, N);
}

}  // namespace

extern "C" lbm_status ffno_forward(ffno_ctx *f, const float *x, float *y, int32_t batch)
{
    if (!f || !x || !y) return ffail(f, LBM_ERR_ARG, "null argument");
    if (batch < 1) return ffail(f, LBM_ERR_ARG, "batch must be positive");
    const ffno_config &c = f->c;
    for (int32_t b0 = 0; b0 < batch; b0 += c.max_batch) {
        const int B = std::min(c.max_batch, batch - b0);
        FCK(cudaMemcpyAsync(f->xin, x + (int64_t)b0 * c.cin * f->N, sizeof(float) * B * c.cin * f->N, cudaMemcpyDefault,
                            f->s));
        forward_impl(f, B);
        FCK(cudaGetLastError());
        FCK(cudaMemcpyAsync(y + (int64_t)b0 * c.cout * f->N, f->y, sizeof(float) * B * c.cout * f->N, cudaMemcpyDefault,
                            f->s));
    }
    if (is_host(y)) FCK(cudaStreamSynchronize(f->s));
    return LBM_OK;
}

extern "C" lbm_status ffno_loss_grad(ffno_ctx *f, const float *x, const float *t, const float *m, int32_t batch,
                                     double *loss)
{
    if (!f || !x || !t || !m) return ffail(f, LBM_ERR_ARG, "null argument");
    const ffno_config &c = f->c;
    if (batch < 1 || batch > c.max_batch) return ffail(f, LBM_ERR_ARG, "batch must lie in [1, max_batch]");
    const int B = batch;
    const int64_t N = f->N;
    FCK(cudaMemcpyAsync(f->xin, x, sizeof(float) * B * c.cin * N, cudaMemcpyDefault, f->s));
    FCK(cudaMemcpyAsync(f->tin, t, sizeof(float) * B * c.cout * N, cudaMemcpyDefault, f->s));
    FCK(cudaMemcpyAsync(f->min, m, sizeof(float) * B * N, cudaMemcpyDefault, f->s));
    forward_impl(f, B);
    k_mse_partial<<<f->nb_loss, TPB, 0, f->s>>>(f->y, f->tin, f->min, c.cout, B, N, f->part);
    k_mse_final<<<1, 32, 0, f->s>>>(f->part, f->nb_loss, c.cout, f->res);
    k_mse_grad<<<grid_for((int64_t)B * c.cout * N), TPB, 0, f->s>>>(f->y, f->tin, f->min, c.cout, B, N, f->res, f->gy);
    backward_impl(f, B);
    FCK(cudaGetLastError());
    double r[2] = {0, 0};
    FCK(cudaMemcpyAsync(r, f->res, sizeof(r), cudaMemcpyDeviceToHost, f->s));
    FCK(cudaStreamSynchronize(f->s));
    if (loss) *loss = r[0];
    return LBM_OK;
}

extern "C" lbm_status ffno_adam_step(ffno_ctx *f, float lr, float b1, float b2, float eps)
{
    if (!f) return LBM_ERR_ARG;
    f->adam_t += 1;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)f->adam_t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)f->adam_t));
    k_adam<<<grid_for(f->np), TPB, 0, f->s>>>(f->params, f->grads, f->m1, f->m2, f->np, lr, b1, b2, eps, c1, c2);
    FCK(cudaGetLastError());
    return LBM_OK;
}
