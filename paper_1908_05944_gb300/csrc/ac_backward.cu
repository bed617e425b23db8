// Differentiation of the filtration values with the combinatorics held fixed.
//
// Every simplex sigma of the complex takes its value from a source simplex s:
// itself when its orthocentre is its closest witness, else the coface whose
// orthocentre is (Section 2.3; the attached case of the proofs of Lemmas 1-2).
// f(sigma) = OrthoSize(s) = min pi(x, b_v0) over the affine set where all
// vertices of s have equal power. With multipliers mu on the equal-power
// constraints the stationarity condition puts the minimiser at
// c = sum_k lambda_k p_k (lambda_0 = 1 - sum mu, lambda_k = mu_k: barycentric
// coordinates of c in aff(s)), and the Lagrangian is sum_k lambda_k pi(c, b_k).
// The envelope theorem then gives
//   dOrthoSize/dp_k = 2 lambda_k (p_k - c),  dOrthoSize/dr_k = -2 r_k lambda_k.
// The gradient is FP64 on the caller's continuous inputs; re-evaluated values
// (for finite-difference checks) use double-double arithmetic.
#include <string.h>

#include <mutex>

#include "ac_internal.cuh"

namespace ac {

struct Ortho {
    double lam[4];
    double c[3];
    double value;
};

// Orthocentre, barycentric coordinates and OrthoSize of K vertices (global input
// indices, ascending) from FP64 centres (n x 3) and radii.
__device__ Ortho ortho_fp64(const double* __restrict__ X, const double* __restrict__ R, const int4& t, int K) {
    Ortho o;
    const int v[4] = {t.x, t.y, t.z, t.w};
    const double p0[3] = {X[3 * v[0]], X[3 * v[0] + 1], X[3 * v[0] + 2]};
    const double w0 = R[v[0]] * R[v[0]];
    double q[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, a[3] = {0, 0, 0};
    for (int k = 1; k < K; k++) {
        double wk = R[v[k]] * R[v[k]];
        for (int c = 0; c < 3; c++) q[k - 1][c] = X[3 * v[k] + c] - p0[c];
        a[k - 1] = q[k - 1][0] * q[k - 1][0] + q[k - 1][1] * q[k - 1][1] + q[k - 1][2] * q[k - 1][2] - wk + w0;
    }
    const int d = K - 1;
    double G[3][3];
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) G[i][j] = q[i][0] * q[j][0] + q[i][1] * q[j][1] + q[i][2] * q[j][2];
    double mu[3] = {0, 0, 0};
    if (d == 1) {
        mu[0] = a[0] / (2.0 * G[0][0]);
    } else if (d == 2) {
        double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        mu[0] = (G[1][1] * a[0] - G[0][1] * a[1]) / (2.0 * det);
        mu[1] = (G[0][0] * a[1] - G[1][0] * a[0]) / (2.0 * det);
    } else if (d == 3) {
        double adj[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
                adj[j][i] = G[r0][c0] * G[r1][c1] - G[r0][c1] * G[r1][c0];
            }
        double det = G[0][0] * adj[0][0] + G[0][1] * adj[1][0] + G[0][2] * adj[2][0];
        for (int i = 0; i < 3; i++) mu[i] = (adj[i][0] * a[0] + adj[i][1] * a[1] + adj[i][2] * a[2]) / (2.0 * det);
    }
    double y[3] = {0, 0, 0};
    for (int k = 0; k < d; k++)
        for (int c = 0; c < 3; c++) y[c] += mu[k] * q[k][c];
    double s = 1.0;
    for (int k = 0; k < d; k++) {
        o.lam[k + 1] = mu[k];
        s -= mu[k];
    }
    o.lam[0] = s;
    for (int c = 0; c < 3; c++) o.c[c] = p0[c] + y[c];
    o.value = y[0] * y[0] + y[1] * y[1] + y[2] * y[2] - w0;
    return o;
}

// Double-double arithmetic (an unevaluated sum hi + lo of two doubles) from the
// error-free transformations TwoSum (Knuth) and TwoProduct via FMA: about 106
// bits, so re-evaluated values of ill-conditioned (flat) simplices stay accurate
// to a few FP64 ulps and central differences with a 1e-6 A step are meaningful.
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_from(double a) { return {a, 0.0}; }

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    return two_sum(p, e);
}

__device__ __forceinline__ dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(b, dd_from(q1)));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(b, dd_from(q2)));
    double q3 = r.hi / b.hi;
    dd q = two_sum(q1, q2);
    return dd_add(q, dd_from(q3));
}

// OrthoSize of K vertices from FP64 centres/radii, evaluated in double-double.
__device__ double orthosize_dd(const double* __restrict__ X, const double* __restrict__ R, const int4& t, int K) {
    const int v[4] = {t.x, t.y, t.z, t.w};
    const dd r0 = dd_from(R[v[0]]);
    const dd w0 = dd_mul(r0, r0);
    if (K == 1) return -w0.hi;
    dd q[3][3], a[3];
    for (int k = 1; k < K; k++) {
        const dd rk = dd_from(R[v[k]]);
        dd sq = dd_from(0.0);
        for (int c = 0; c < 3; c++) {
            q[k - 1][c] = two_sum(X[3 * v[k] + c], -X[3 * v[0] + c]);
            sq = dd_add(sq, dd_mul(q[k - 1][c], q[k - 1][c]));
        }
        a[k - 1] = dd_add(dd_sub(sq, dd_mul(rk, rk)), w0);
    }
    auto dot = [](const dd* x, const dd* y) {
        return dd_add(dd_add(dd_mul(x[0], y[0]), dd_mul(x[1], y[1])), dd_mul(x[2], y[2]));
    };
    dd num, den;
    if (K == 2) {
        dd D = dot(q[0], q[0]);
        num = dd_mul(a[0], a[0]);
        den = dd_mul(dd_from(4.0), D);
    } else if (K == 3) {
        dd g11 = dot(q[0], q[0]), g22 = dot(q[1], q[1]), g12 = dot(q[0], q[1]);
        dd det = dd_sub(dd_mul(g11, g22), dd_mul(g12, g12));
        dd n1 = dd_sub(dd_mul(g22, a[0]), dd_mul(g12, a[1]));
        dd n2 = dd_sub(dd_mul(g11, a[1]), dd_mul(g12, a[0]));
        num = dd_add(dd_mul(n1, a[0]), dd_mul(n2, a[1]));
        den = dd_mul(dd_from(4.0), det);
    } else {
        dd C[3][3];
        for (int k = 0; k < 3; k++) {
            const dd* b = q[(k + 1) % 3];
            const dd* e = q[(k + 2) % 3];
            C[k][0] = dd_sub(dd_mul(b[1], e[2]), dd_mul(b[2], e[1]));
            C[k][1] = dd_sub(dd_mul(b[2], e[0]), dd_mul(b[0], e[2]));
            C[k][2] = dd_sub(dd_mul(b[0], e[1]), dd_mul(b[1], e[0]));
        }
        dd D = dot(q[0], C[0]);
        dd N[3];
        for (int c = 0; c < 3; c++)
            N[c] = dd_add(dd_add(dd_mul(a[0], C[0][c]), dd_mul(a[1], C[1][c])), dd_mul(a[2], C[2][c]));
        num = dot(N, N);
        den = dd_mul(dd_from(4.0), dd_mul(D, D));
    }
    dd f = dd_sub(dd_div(num, den), w0);
    return f.hi + f.lo;
}

// OrthoSize of K vertices in single precision throughout: offsets q_k =
// p_k - p_0 and squared radii from the quantised atoms (exact in FP32), then
// a_k, the Gram matrix, its solve and |y|^2 - w_0 rounded to FP32 at every
// operation. Not used by the build: it measures what FP32 arithmetic would
// do to the filtration values.
__device__ float orthosize_f32(const int4* __restrict__ P, const int4& t, int K) {
    const int v[4] = {t.x, t.y, t.z, t.w};
    const int4 p0 = P[v[0]];
    const float s = 1.0f / 1024.0f, s2 = 1.0f / 1048576.0f;
    const float w0 = (float)p0.w * s2;
    if (K == 1) return -w0;
    float q[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, a[3] = {0.f, 0.f, 0.f};
    for (int k = 1; k < K; k++) {
        const int4 pk = P[v[k]];
        q[k - 1][0] = (float)(pk.x - p0.x) * s;
        q[k - 1][1] = (float)(pk.y - p0.y) * s;
        q[k - 1][2] = (float)(pk.z - p0.z) * s;
        a[k - 1] = q[k - 1][0] * q[k - 1][0] + q[k - 1][1] * q[k - 1][1] + q[k - 1][2] * q[k - 1][2] -
                   (float)pk.w * s2 + w0;
    }
    const int d = K - 1;
    float G[3][3];
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) G[i][j] = q[i][0] * q[j][0] + q[i][1] * q[j][1] + q[i][2] * q[j][2];
    float mu[3] = {0.f, 0.f, 0.f};
    if (d == 1) {
        mu[0] = a[0] / (2.0f * G[0][0]);
    } else if (d == 2) {
        const float det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        mu[0] = (G[1][1] * a[0] - G[0][1] * a[1]) / (2.0f * det);
        mu[1] = (G[0][0] * a[1] - G[1][0] * a[0]) / (2.0f * det);
    } else {
        float adj[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
                adj[j][i] = G[r0][c0] * G[r1][c1] - G[r0][c1] * G[r1][c0];
            }
        const float det = G[0][0] * adj[0][0] + G[0][1] * adj[1][0] + G[0][2] * adj[2][0];
        for (int i = 0; i < 3; i++) mu[i] = (adj[i][0] * a[0] + adj[i][1] * a[1] + adj[i][2] * a[2]) / (2.0f * det);
    }
    float y[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < d; k++)
        for (int c = 0; c < 3; c++) y[c] += mu[k] * q[k][c];
    return y[0] * y[0] + y[1] * y[1] + y[2] * y[2] - w0;
}

struct Rows4 {
    const int4* G[4];
};

__global__ void k_eval_f32(const int4* __restrict__ P, const int8_t* __restrict__ sdim, const int64_t* __restrict__ sidx,
                           int64_t m, Rows4 rows, float* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int d = sdim[j];
    out[j] = orthosize_f32(P, rows.G[d][sidx[j]], d + 1);
}

int eval_filtration_f32(ac_ctx* c, float* const f_out[4], cudaStream_t s) {
    Rows4 rows;
    for (int d = 0; d < 4; d++) rows.G[d] = c->Gbuf[d].as<int4>();
    for (int d = 0; d < 4; d++) {
        const int64_t m = c->K[d].count;
        if (!f_out[d] || m == 0) continue;
        k_eval_f32<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(c->P.as<int4>(), c->K[d].src_dim.as<int8_t>(),
                                                               c->K[d].src_idx.as<int64_t>(), m, rows, f_out[d]);
        AC_LAUNCHED();
    }
    AC_CUDA(cudaStreamSynchronize(s));
    return AC_OK;
}

__global__ void k_eval(const double* __restrict__ X, const double* __restrict__ R, const int8_t* __restrict__ sdim,
                       const int64_t* __restrict__ sidx, int64_t m, const int4* const* __restrict__ G,
                       double* __restrict__ out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int d = sdim[j];
    const int4 t = G[d][sidx[j]];
    out[j] = orthosize_dd(X, R, t, d + 1);
}

__global__ void k_backward(const double* __restrict__ X, const double* __restrict__ R, const int8_t* __restrict__ sdim,
                           const int64_t* __restrict__ sidx, int64_t m, const int4* const* __restrict__ G,
                           const double* __restrict__ w, double* __restrict__ dX, double* __restrict__ dR) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double wj = w[j];
    if (wj == 0.0) return;
    const int d = sdim[j];
    const int4 t = G[d][sidx[j]];
    const Ortho o = ortho_fp64(X, R, t, d + 1);
    const int v[4] = {t.x, t.y, t.z, t.w};
    for (int k = 0; k <= d; k++) {
        const int a = v[k];
        const double l2 = 2.0 * wj * o.lam[k];
        for (int c = 0; c < 3; c++) atomicAdd(&dX[3 * a + c], l2 * (X[3 * a + c] - o.c[c]));
        atomicAdd(&dR[a], -l2 * R[a]);
    }
}

static int gtable(ac_ctx* c, DevBuf& tab, cudaStream_t s) {
    const int4* h[4];
    for (int d = 0; d < 4; d++) h[d] = c->Gbuf[d].as<int4>();
    AC_TRY(tab.reserve(sizeof(h), s));
    AC_CUDA(cudaMemcpyAsync(tab.p, h, sizeof(h), cudaMemcpyHostToDevice, s));
    return AC_OK;
}

int eval_filtration(ac_ctx* c, const double* centres, const double* radii, double* const f_out[4], cudaStream_t s) {
    AC_TRY(gtable(c, c->scratch[5], s));
    for (int d = 0; d < 4; d++) {
        const int64_t m = c->K[d].count;
        if (!f_out[d] || m == 0) continue;
        k_eval<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(centres, radii, c->K[d].src_dim.as<int8_t>(),
                                                           c->K[d].src_idx.as<int64_t>(), m,
                                                           c->scratch[5].as<const int4*>(), f_out[d]);
        AC_LAUNCHED();
    }
    AC_CUDA(cudaStreamSynchronize(s));
    return AC_OK;
}

// ---------------------------------------------------------------------------
// ac_backward: the same gradient, with every sum taken in a fixed order, so
// that repeated calls give bit-identical results (no floating-point atomics).
//
// Sum over the simplices sigma of w_sigma * dOrthoSize(src(sigma)): grouped by
// source, each source s contributes W_s * dOrthoSize(s), W_s the sum of the
// weights of the simplices whose source it is. An attached simplex takes its
// source from its parent, the coface its value came from (the build's
// coface passes keep, for every coface, the rows of its attached facets, and
// for every attached row its parent), and an unattached one is its own
// source. So:
//   1. k_weights_up, dimension 0 to 3, one thread per row: W'(sigma) =
//      w(sigma) + the W' of the attached facets whose parent sigma is, in
//      facet order. An unattached row's W' is its W_s; an attached row hands
//      its W' up and is no source.
//   2. k_contrib, one thread per unattached row with W_s != 0: the
//      orthocentre and barycentric coordinates of s, and for each vertex k of
//      s the contribution (2 W_s lambda_k (p_k - c), -2 W_s lambda_k r_k).
//   3. k_gather_atoms, one warp per atom a: the contributions of the rows
//      containing a, summed per lane and then over the lanes by a fixed tree.
//      Every vertex of a simplex of the complex has a grown ball meeting a's,
//      so the first (smallest) vertex of a row containing a is a or one of
//      a's neighbours with a smaller input index: lane t takes neighbour t
//      (and lane 0 a itself first), every list, every row of that first vertex.

struct BackArgs {
    const double* X;         // centres (n x 3), input order
    const double* R;         // radii
    const int4* G[4];        // rows per dimension, global input indices
    const int64_t* v0[4];    // rows with first vertex g start at v0[d][g] (n + 1)
    const uint8_t* att[4];   // attached flags
    const double* w[4];      // dL/df per row (NULL: zero)
    double* Wp[4];           // W' per row (pass 1)
    const int64_t* frows[3]; // frows[d]: rows of the attached facets (dim d) of each coface (dim d + 1), or -1
    const unsigned long long* parent[3];  // parent[d][r]: the coface (row of dim d + 1) of attached row r of dim d
    double4* C[4];           // per row, per vertex: (dL/dp, dL/dr) contributions (pass 2)
    int64_t rows[4];
    const int32_t* rank;     // input index -> sorted position
    const int32_t* order;    // sorted position -> input index
    const int64_t* nb_off;   // neighbour rows (as in the per-atom pass)
    const int32_t* nb;
    int nb_stride;
    int64_t n;
};

__global__ void k_weights_up(BackArgs A, int d) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.rows[d]) return;
    double W = A.w[d] ? A.w[d][j] : 0.0;
    if (d >= 1 && A.frows[d - 1]) {
        const int64_t* fr = A.frows[d - 1] + j * (d + 1);
        for (int drop = 0; drop <= d; drop++) {
            const int64_t r = fr[drop];
            if (r >= 0 && A.parent[d - 1][r] == (unsigned long long)j) W += A.Wp[d - 1][r];
        }
    }
    A.Wp[d][j] = W;
}

__global__ void k_contrib(BackArgs A, int d) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.rows[d]) return;
    double4* out = A.C[d] + j * (d + 1);
    const double W = A.att[d][j] ? 0.0 : A.Wp[d][j];
    if (W == 0.0) {
        for (int k = 0; k <= d; k++) out[k] = make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const int4 g = A.G[d][j];
    const int v[4] = {g.x, g.y, g.z, g.w};
    const Ortho o = ortho_fp64(A.X, A.R, g, d + 1);
    for (int k = 0; k <= d; k++) {
        const int64_t a = v[k];
        const double l2 = 2.0 * W * o.lam[k];
        out[k] = make_double4(l2 * (A.X[3 * a] - o.c[0]), l2 * (A.X[3 * a + 1] - o.c[1]), l2 * (A.X[3 * a + 2] - o.c[2]),
                              -l2 * A.R[a]);
    }
}

constexpr int GATHER_WARPS = 4;

__global__ void __launch_bounds__(GATHER_WARPS * 32) k_gather_atoms(BackArgs A, double* __restrict__ dX,
                                                                     double* __restrict__ dR) {
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * GATHER_WARPS + (threadIdx.x >> 5);
    if (a >= A.n) return;
    const int ia = A.rank[a];
    const int64_t off = A.nb_stride ? (int64_t)ia * A.nb_stride : A.nb_off[ia];
    const int m = A.nb_stride ? (int)A.nb_off[ia] : (int)(A.nb_off[ia + 1] - off);
    double gx = 0.0, gy = 0.0, gz = 0.0, gr = 0.0;
    for (int t = lane - 1; t < m; t += 32) {
        const int64_t b = t < 0 ? a : (int64_t)A.order[A.nb[off + t]];
        if (t >= 0 && b >= a) continue;
        for (int d = 0; d < 4; d++) {
            for (int64_t r = A.v0[d][b]; r < A.v0[d][b + 1]; r++) {
                const int4 g = A.G[d][r];
                const int k = g.x == a ? 0 : (d >= 1 && g.y == a) ? 1 : (d >= 2 && g.z == a) ? 2 : (d >= 3 && g.w == a) ? 3 : -1;
                if (k < 0) continue;
                const double4 q = A.C[d][r * (d + 1) + k];
                gx += q.x;
                gy += q.y;
                gz += q.z;
                gr += q.w;
            }
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {  // a fixed tree: the same additions in the same order every call
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
    }
    if (lane == 0) {
        dX[3 * a] = gx;
        dX[3 * a + 1] = gy;
        dX[3 * a + 2] = gz;
        dR[a] = gr;
    }
}

int backward(ac_ctx* c, const double* const dldf[4], double* dc, double* dr, cudaStream_t s) {
    const int64_t n = c->n;
    if (n == 0) return AC_OK;
    BackArgs A;
    memset(&A, 0, sizeof(A));
    A.X = c->centres.as<double>();
    A.R = c->radii.as<double>();
    size_t wrows = 0, crows = 0;
    for (int d = 0; d < 4; d++) {
        wrows += (size_t)c->K[d].count;
        crows += (size_t)c->K[d].count * (d + 1);
    }
    const size_t wbytes = ((wrows > 0 ? wrows : 1) * sizeof(double) + 255) & ~(size_t)255;
    AC_TRY(c->scratch[3].reserve(wbytes + (crows > 0 ? crows : 1) * sizeof(double4), s));
    double* Wbuf = c->scratch[3].as<double>();
    double4* Cbuf = reinterpret_cast<double4*>(static_cast<char*>(c->scratch[3].p) + wbytes);
    for (int d = 0; d < 4; d++) {
        const int64_t m = c->K[d].count;
        A.G[d] = c->Gbuf[d].as<int4>();
        A.v0[d] = c->K[d].v0_off.as<int64_t>();
        A.att[d] = c->K[d].attached.as<uint8_t>();
        A.w[d] = m > 0 ? dldf[d] : nullptr;
        A.Wp[d] = Wbuf;
        A.C[d] = Cbuf;
        A.rows[d] = m;
        Wbuf += m;
        Cbuf += m * (d + 1);
        if (d < 3) {
            const bool cof = c->K[d + 1].count > 0;  // the coface passes ran: frows[d], fargs[d] hold this build's
            A.frows[d] = cof ? c->frows[d].as<int64_t>() : nullptr;
            A.parent[d] = cof ? c->fargs[d].as<unsigned long long>() : nullptr;
        }
    }
    A.rank = c->rank.as<int32_t>();
    A.order = c->order.as<int32_t>();
    A.nb_off = c->nb_cnt.as<int64_t>();
    A.nb = c->nb.as<int32_t>();
    A.nb_stride = c->nb_stride;
    A.n = n;
    for (int d = 0; d < 4; d++) {
        const int64_t m = A.rows[d];
        if (m == 0) continue;
        k_weights_up<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(A, d);
        AC_LAUNCHED();
    }
    for (int d = 0; d < 4; d++) {
        const int64_t m = A.rows[d];
        if (m == 0) continue;
        k_contrib<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(A, d);
        AC_LAUNCHED();
    }
    k_gather_atoms<<<(unsigned)((n + GATHER_WARPS - 1) / GATHER_WARPS), GATHER_WARPS * 32, 0, s>>>(A, dc, dr);
    AC_LAUNCHED();
    AC_CUDA(cudaStreamSynchronize(s));
    return AC_OK;
}

// ---------------------------------------------------------------------------
// ac_backward_noalloc: the gradient without any device allocation.
//
// ac_backward sums in a fixed order with per-simplex scratch it allocates.
// Callers that cannot allocate device memory (for example inside a training
// step whose memory belongs to another allocator, or a service with a fixed
// device memory budget) use this entry point instead: it runs k_backward (one
// thread per simplex, FP64 atomics), whose only scratch is the table of the
// four per-dimension source-list pointers it reads, and that table lives in
// the static array below, which every GPU that loads the library holds until
// the process exits. Maximum: NOALLOC_TABLE_ENTRIES = 4 pointers (one per
// dimension 0..3), 32 bytes in a 256-byte-aligned array. Every call overwrites
// the whole table before its kernels read it, so nothing in it has to start at
// zero; calls that overlap on the GPU (other streams, other host threads)
// share the one table and race. The cached device address of the table does
// not survive a cudaDeviceReset.
constexpr int NOALLOC_TABLE_ENTRIES = 4;
static __device__ __align__(256) const int4* g_noalloc_table[NOALLOC_TABLE_ENTRIES];

// Device addresses of g_noalloc_table, looked up once per device with that
// device current (the host-side name is only a stand-in).
constexpr int NOALLOC_MAX_DEVICES = 64;
static const int4** g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static int noalloc_table(const int4*** out) {
    int dev = 0;
    AC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(AC_ERR_INVALID_ARG, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_table);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_table)", __FILE__, __LINE__);
        g_noalloc_addr[dev] = (const int4**)ptr;
    }
    *out = g_noalloc_addr[dev];
    return AC_OK;
}

int backward_noalloc(ac_ctx* c, const double* const dldf[4], double* dc, double* dr, cudaStream_t s) {
    const int lists = 4;
    if (lists > NOALLOC_TABLE_ENTRIES) return fail(AC_ERR_CAPACITY, "more simplex lists than the static table holds");
    const int4** table = nullptr;
    AC_TRY(noalloc_table(&table));
    const int4* h[NOALLOC_TABLE_ENTRIES];
    for (int d = 0; d < lists; d++) h[d] = c->Gbuf[d].as<int4>();
    AC_CUDA(cudaMemcpyAsync(table, h, sizeof(h), cudaMemcpyHostToDevice, s));
    const int64_t n = c->n;
    AC_CUDA(cudaMemsetAsync(dc, 0, (size_t)(n > 0 ? n : 0) * 3 * sizeof(double), s));
    AC_CUDA(cudaMemsetAsync(dr, 0, (size_t)(n > 0 ? n : 0) * sizeof(double), s));
    for (int d = 0; d < lists; d++) {
        const int64_t m = c->K[d].count;
        if (!dldf[d] || m == 0) continue;
        k_backward<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(c->centres.as<double>(), c->radii.as<double>(),
                                                               c->K[d].src_dim.as<int8_t>(), c->K[d].src_idx.as<int64_t>(),
                                                               m, table, dldf[d], dc, dr);
        AC_LAUNCHED();
    }
    AC_CUDA(cudaStreamSynchronize(s));
    return AC_OK;
}

}  // namespace ac
