// The per-atom pass: potential simplices (Section 4.3, Step 1 of Section 3.1)
// and their AC2 tests (Section 4.4, Steps 2-5), fused in one kernel.
//
// Ownership. A simplex is owned by its vertex with the lowest sorted position
// i. One warp handles one owner at a time and works entirely inside L(i), the
// list of i's neighbours (atoms whose grown balls meet i's, ac_grid.cu), held
// in shared memory as exact integer offsets q_x = P_x - P_i together with
// a_x = |q_x|^2 - W_x + W_i. Bitmasks over positions in L(i) (WORDS 32-bit
// words, so |L(i)| <= 32 * WORDS) carry every relation:
//   up       positions x > i with edge (i,x) in Sigma_ortho^1 (edge AC3 exact)
//   M[p]     positions adjacent to p (grown balls meet), for p in up
//   T[p]     positions k > p with triangle (i,p,k) in Sigma_ortho^2
// Potential triangles are pairs (p,k), k in M[p] & up, k > p; potential
// tetrahedra are (p,k,l) with l in T[p] & T[k]. Monotonicity of OrthoSize
// (Section 4.3) makes this complete: every face of a simplex in Sigma_ortho is
// in Sigma_ortho. AC3 is then decided exactly for each candidate.
//
// AC2 at the orthocentre c of sigma. Every ball x that violates it (ties
// included) has pi(c, b_x) <= OrthoSize(sigma) <= alpha, so its grown ball
// contains c, as does every vertex's; x is therefore adjacent to all vertices:
// the candidates are M[p] & M[k] & M[l] (all of L(i) for the vertex i itself),
// not a stencil of cells around c. For each candidate,
//   Delta_x = pi(c, b_x) - pi(c, b_i) = a_x - 2 q_x . y,  y = c - P_i,
// and AC2 fails iff some Delta_x < 0 (ties: symbolic perturbation below).
//
// Predicate cascade (precision AC_PRECISION_FILTERED). y is formed from exact
// integer minors (tetrahedron: y = N / (2D), N = a1 (q2 x q3) + a2 (q3 x q1) +
// a3 (q1 x q2), D = det(q1, q2, q3); triangle: y = mu1 q1 + mu2 q2 with
// mu = adj(G) a / (2 det G), G the Gram matrix), rounded once to FP32, and
// Delta is evaluated in FP32 with a static forward error bound:
//   |fl(Delta) - Delta| <= u|fl(Delta)|(1+u) + u|a_x| + 2 gamma_3 |q_x||y~|
//                          + 2 |q_x| |y~ - y|
// with u = 2^-24, gamma_3 = 3u/(1-3u), |q_x| <= 2h (x is a neighbour of i),
// |y| <= h (OrthoSize <= alpha gives |y|^2 <= W_i + A <= h^2) and
// |a_x| <= 4h^2 + max W. For a tetrahedron |y~_c - y_c| <= 4.0001u |y_c|
// (three roundings of N, D and one of the reciprocal, one of the product);
// for a triangle the bound is accumulated per triangle from |mu~| |q|.
// Undecided cases are recomputed in FP64 with the same bound at u = 2^-53,
// then decided exactly in 128-bit integers. AC_PRECISION_PLAIN_FP64 starts at
// the FP64 level. Edges and vertices are decided in exact 64-bit integers.
//
// Ties (Section 2, symbolic perturbation): squared radii W_k + eps_k with
// eps_k falling steeply in the INPUT index k. Delta_x is affine in the
// weights; its coefficient on W_x is -|D| < 0, on W_v (v a vertex of sigma)
// it is |D| lambda_v(x), lambda the affine coordinates of x (projected onto
// aff(sigma)) in the vertices of sigma. When Delta_x = 0 the coefficient of the
// smallest input index with a non-zero coefficient gives the sign.
//   tetrahedron: D lambda_k = det(Q with row k replaced by q_x) = q_x . C_k
//   triangle:    detG lambda = adj(G) (q_1.q_x, q_2.q_x)
//   edge:        D lambda_1 = q.q_x
// and lambda_i = 1 - sum of the others. Exact 64-bit integers.
#include "ac_internal.cuh"

namespace ac {

constexpr unsigned FULL = 0xffffffffu;
constexpr int STAGE = 64;

template <int WORDS>
struct WarpSmem {
    static constexpr int M = 32 * WORDS;
    int4 q[M];      // (qx, qy, qz, a_x) exact
    float4 qf[M];   // the same in FP32 (a_x rounded)
    int s[M];       // W_x + A
    int gid[M];     // input index
    int idx[M];     // sorted position
    unsigned Mrow[M][WORDS];
    unsigned Trow[M][WORDS];
    unsigned up[WORDS];
    unsigned char uplist[M];
    int n_up;
    int n_tet, n_tri, n_edge;
    int4 st_tet[STAGE];
    int4 st_tri[STAGE];
    int2 st_edge[STAGE];
};

struct LocalArgs {
    const int4* Ps;
    const int32_t* order;
    const int64_t* nb_off;
    const int32_t* nb;
    int64_t n;
    PredConst pc;
    // FP32/FP64 triangle thresholds: E = (k0 + k1 * e) where e bounds |y~ - y|
    float tri_k0_32, tri_k1_32;
    double tri_k0_64, tri_k1_64;
    float tet_eps32;
    double tet_eps64;
    int4* tet_out;
    int64_t cap_tet;
    int4* tri_out;
    int64_t cap_tri;
    int2* edge_out;
    int64_t cap_edge;
    uint8_t* vert_pass;
    int4* cand3;
    int4* cand2;
    int2* cand1;
    int64_t cap_cand[4];
    DevCounters* cnt;
};

struct LaneCounts {
    unsigned tet[3], tri[3], edge;
    unsigned ac3[4];
    unsigned cand[4];
};

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// position of the r-th (0-based) set bit of m; requires r < popc(m)
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        unsigned low = (1u << w) - 1u;
        int c = __popc(m & low);
        if (r >= c) {
            r -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// Warp-cooperative expansion: each lane holds (tag, mask); f(valid, tag, bit) is
// called by every lane, 32 (tag, bit) pairs per round, until all set bits of
// all lanes' masks have been visited.
template <int WORDS, class F>
__device__ __forceinline__ void warp_expand(const int lane, const unsigned (&mask)[WORDS], const int tag, F&& f) {
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < WORDS; w++) cnt += __popc(mask[w]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - cnt;
    for (int base = 0; base < total; base += 32) {
        const int j = base + lane;
        int o = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            int cand = o + step;
            int e = __shfl_sync(FULL, excl, cand & 31);
            if (cand < 32 && e <= j) o = cand;
        }
        int r = j - __shfl_sync(FULL, excl, o);
        int otag = __shfl_sync(FULL, tag, o);
        int bit = -1;
#pragma unroll
        for (int w = 0; w < WORDS; w++) {
            unsigned mw = __shfl_sync(FULL, mask[w], o);
            int pc = __popc(mw);
            if (bit < 0 && j < total) {
                if (r < pc) bit = 32 * w + nth_set_bit(mw, r);
                else r -= pc;
            }
        }
        f(j < total, otag, bit);
    }
}

template <class T>
__device__ void stage_flush(const int lane, T* stage, int* n_stage, T* out, unsigned long long* counter, int64_t cap,
                            unsigned* err, unsigned bit) {
    __syncwarp();
    const int cnt = *n_stage;
    if (cnt > 0) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, (unsigned long long)cnt);
        base = __shfl_sync(FULL, base, 0);
        for (int j = lane; j < cnt; j += 32)
            if ((int64_t)(base + j) < cap) out[base + j] = stage[j];
        if (lane == 0 && (int64_t)(base + cnt) > cap) atomicOr(err, bit);
    }
    __syncwarp();
    if (lane == 0) *n_stage = 0;
    __syncwarp();
}

template <class T>
__device__ __forceinline__ void stage_push(const int lane, bool want, const T& item, T* stage, int* n_stage, T* out,
                                           unsigned long long* counter, int64_t cap, unsigned* err, unsigned bit) {
    unsigned b = __ballot_sync(FULL, want);
    if (b == 0) return;
    const int k = __popc(b);
    if (*n_stage + k > STAGE) stage_flush(lane, stage, n_stage, out, counter, cap, err, bit);
    const int cur = *n_stage;
    if (want) stage[cur + __popc(b & lanemask_lt())] = item;
    __syncwarp();
    if (lane == 0) *n_stage = cur + k;
    __syncwarp();
}

template <class T>
__device__ __forceinline__ void append_direct(bool want, const T& item, T* out, unsigned long long* counter, int64_t cap,
                                              unsigned* err) {
    unsigned b = __ballot_sync(FULL, want);
    if (b == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(b) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(b));
    base = __shfl_sync(FULL, base, leader);
    if (want) {
        unsigned long long slot = base + __popc(b & lanemask_lt());
        if ((int64_t)slot < cap) out[slot] = item;
        else atomicOr(err, DERR_OVF_CAND);
    }
}

// smallest input index among the candidates with a non-zero coefficient
// decides the sign of a Delta that is exactly zero. Returns true if Delta_eps < 0.
__device__ __forceinline__ bool sos_violates(int nv, const int* g, const long long* coef, int gx) {
    int best = gx;
    int sign = -1;  // the test ball's own coefficient is negative
    for (int k = 0; k < nv; k++)
        if (coef[k] != 0 && g[k] < best) {
            best = g[k];
            sign = coef[k] > 0 ? 1 : -1;
        }
    return sign < 0;
}

__device__ __forceinline__ i128 mul64x64(long long a, long long b) { return (i128)a * (i128)b; }

// ---------------------------------------------------------------------------

template <int WORDS>
__global__ void __launch_bounds__(256) k_local(LocalArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = WarpSmem<WORDS>;
    constexpr int MAXM = SM::M;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    SM& S = reinterpret_cast<SM*>(smem_raw)[wib];
    DevCounters* cnt = A.cnt;
    const PredConst& pc = A.pc;
    const int64_t Aq = pc.A;
    const bool filtered = pc.precision == AC_PRECISION_FILTERED;
    LaneCounts lc;
    memset(&lc, 0, sizeof(lc));
    if (lane == 0) {
        S.n_tet = 0;
        S.n_tri = 0;
        S.n_edge = 0;
    }
    __syncwarp();

    for (;;) {
        long long i_ll = 0;
        if (lane == 0) i_ll = (long long)atomicAdd(&cnt->work_next, 1ull);
        i_ll = __shfl_sync(FULL, i_ll, 0);
        if (i_ll >= A.n) break;
        const int i = (int)i_ll;
        const int4 Pi = A.Ps[i];
        const int Wi = Pi.w;
        const long long si = (long long)Wi + Aq;
        const int gi = A.order[i];
        const int64_t off = A.nb_off[i];
        const int m = (int)(A.nb_off[i + 1] - off);
        if (si < 0) {
            if (lane == 0) A.vert_pass[i] = 0;
            continue;
        }
        if (m > MAXM) {
            if (lane == 0) atomicOr(&cnt->err, DERR_DEGREE);
            continue;
        }

        // ---- phase A: load L(i); upper edges with exact edge AC3 ------------
        unsigned vert_bad = 0;
#pragma unroll
        for (int w = 0; w < WORDS; w++) {
            const int e = 32 * w + lane;
            bool upper = false;
            if (e < m) {
                const int x = A.nb[off + e];
                const int4 o = A.Ps[x];
                const int qx = o.x - Pi.x, qy = o.y - Pi.y, qz = o.z - Pi.z;
                const int D = qx * qx + qy * qy + qz * qz;  // <= 3 * 2^26
                const int ax = D - o.w + Wi;
                S.q[e] = make_int4(qx, qy, qz, ax);
                S.qf[e] = make_float4((float)qx, (float)qy, (float)qz, (float)ax);
                S.s[e] = (int)((long long)o.w + Aq);
                const int gx = A.order[x];
                S.gid[e] = gx;
                S.idx[e] = x;
                // vertex AC2 at p_i (Step 5): Delta_x = a_x; tie -> smaller input index wins
                if (ax < 0 || (ax == 0 && gx < gi)) vert_bad = 1;
                if (x > i) {
                    // edge AC3: (D + W_i - W_x)^2 <= 4 D (W_i + A)
                    const long long a = (long long)D + Wi - o.w;
                    upper = a * a <= 4ll * D * si;
                    lc.ac3[1]++;
                }
            }
            const unsigned b = __ballot_sync(FULL, upper);
            if (lane == 0) S.up[w] = b;
        }
        vert_bad = __any_sync(FULL, vert_bad);
        if (lane == 0) A.vert_pass[i] = vert_bad ? 0 : 1;
        __syncwarp();
        // list of upper positions
        {
            int base = 0;
#pragma unroll
            for (int w = 0; w < WORDS; w++) {
                const unsigned b = S.up[w];
                if ((b >> lane) & 1u) S.uplist[base + __popc(b & lanemask_lt())] = (unsigned char)(32 * w + lane);
                base += __popc(b);
            }
            if (lane == 0) S.n_up = base;
            lc.cand[1] += lane == 0 ? base : 0;
        }
        __syncwarp();
        const int n_up = S.n_up;
        if (pc.keep_candidates) {
            for (int r0 = 0; r0 < n_up; r0 += 32) {
                const bool ok = r0 + lane < n_up;
                const int p = ok ? S.uplist[r0 + lane] : 0;
                append_direct(ok, make_int2(i, ok ? S.idx[p] : 0), A.cand1, &cnt->n_cand_out[1], A.cap_cand[1], &cnt->err);
            }
        }

        // ---- phase B: adjacency rows M[p] for p in up -----------------------
        for (int r = 0; r < n_up; r++) {
            const int p = S.uplist[r];
            const int4 qp = S.q[p];
            const long long sp = S.s[p];
#pragma unroll
            for (int w = 0; w < WORDS; w++) {
                const int e = 32 * w + lane;
                bool adj = false;
                if (e < m && e != p) {
                    const int4 qe = S.q[e];
                    const int dx = qe.x - qp.x, dy = qe.y - qp.y, dz = qe.z - qp.z;  // |.| <= 2^14
                    const long long D = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
                    const long long se = S.s[e];
                    const long long t = D - sp - se;
                    adj = t <= 0 || t * t <= 4 * sp * se;
                }
                const unsigned b = __ballot_sync(FULL, adj);
                if (lane == 0) {
                    S.Mrow[p][w] = b;
                    S.Trow[p][w] = 0u;
                }
            }
        }
        __syncwarp();

        // ---- phase C: triangles (i,p,k): AC3 exact, then AC2 -----------------
        for (int r0 = 0; r0 < n_up; r0 += 32) {
            const bool rowok = r0 + lane < n_up;
            const int p = rowok ? S.uplist[r0 + lane] : 0;
            unsigned mask[WORDS];
#pragma unroll
            for (int w = 0; w < WORDS; w++) {
                unsigned above;
                if (32 * w + 31 <= p) above = 0u;
                else if (32 * w > p) above = FULL;
                else above = ~((2u << (p & 31)) - 1u);
                mask[w] = rowok ? (S.Mrow[p][w] & S.up[w] & above) : 0u;
            }
            warp_expand<WORDS>(lane, mask, p, [&](bool valid, int pp, int kk) {
                bool in_sigma = false, pass = false;
                if (valid) {
                    const int4 q1 = S.q[pp], q2 = S.q[kk];
                    const long long g11 = (long long)q1.x * q1.x + (long long)q1.y * q1.y + (long long)q1.z * q1.z;
                    const long long g22 = (long long)q2.x * q2.x + (long long)q2.y * q2.y + (long long)q2.z * q2.z;
                    const long long g12 = (long long)q1.x * q2.x + (long long)q1.y * q2.y + (long long)q1.z * q2.z;
                    const long long detG = g11 * g22 - g12 * g12;
                    lc.ac3[2]++;
                    if (detG > 0) {
                        const long long a1 = q1.w, a2 = q2.w;
                        const long long n1 = g22 * a1 - g12 * a2, n2 = g11 * a2 - g12 * a1;
                        const i128 na = mul64x64(n1, a1) + mul64x64(n2, a2);
                        in_sigma = na <= (i128)(4 * detG) * (i128)si;
                    }
                    if (in_sigma) {
                        lc.cand[2]++;
                        atomicOr(&S.Trow[pp][kk >> 5], 1u << (kk & 31));
                        // AC2 at the triangle's orthocentre
                        const long long a1 = q1.w, a2 = q2.w;
                        const long long n1 = g22 * a1 - g12 * a2, n2 = g11 * a2 - g12 * a1;
                        float y32[3] = {0.f, 0.f, 0.f}, E32 = 0.f;
                        double y64[3] = {0.0, 0.0, 0.0}, E64 = 0.0;
                        bool have64 = false;
                        if (filtered) {
                            const float rd = __frcp_rn(2.0f * __ll2float_rn(detG));
                            const float m1 = __fmul_rn(__ll2float_rn(n1), rd), m2 = __fmul_rn(__ll2float_rn(n2), rd);
                            const float q1f[3] = {(float)q1.x, (float)q1.y, (float)q1.z};
                            const float q2f[3] = {(float)q2.x, (float)q2.y, (float)q2.z};
                            float e = 0.f;
#pragma unroll
                            for (int c = 0; c < 3; c++) {
                                y32[c] = __fmaf_rn(m1, q1f[c], __fmul_rn(m2, q2f[c]));
                                e = __fmaf_ru(fabsf(m1), fabsf(q1f[c]), __fmaf_ru(fabsf(m2), fabsf(q2f[c]), e));
                            }
                            e = __fmul_ru(e, 6.05f * 5.9604645e-8f);
                            E32 = __fmaf_ru(A.tri_k1_32, e, A.tri_k0_32);
                        }
                        auto make64 = [&]() {
                            const double rd = 1.0 / (2.0 * (double)detG);
                            const double m1 = (double)n1 * rd, m2 = (double)n2 * rd;
                            const double q1d[3] = {(double)q1.x, (double)q1.y, (double)q1.z};
                            const double q2d[3] = {(double)q2.x, (double)q2.y, (double)q2.z};
                            double e = 0.0;
                            for (int c = 0; c < 3; c++) {
                                y64[c] = fma(m1, q1d[c], m2 * q2d[c]);
                                e += fabs(m1) * fabs(q1d[c]) + fabs(m2) * fabs(q2d[c]);
                            }
                            e *= 6.05 * 1.1102230246251565e-16 * (1.0 + 1e-10);
                            E64 = (A.tri_k0_64 + A.tri_k1_64 * e) * (1.0 + 1e-10);
                            have64 = true;
                        };
                        if (!filtered) make64();
                        unsigned V[WORDS];
#pragma unroll
                        for (int w = 0; w < WORDS; w++) V[w] = S.Mrow[pp][w] & S.Mrow[kk][w];
                        bool violated = false;
#pragma unroll
                        for (int w = 0; w < WORDS; w++) {
                            unsigned b = V[w];
                            while (b && !violated) {
                                const int x = 32 * w + __ffs(b) - 1;
                                b &= b - 1;
                                int decided = 0;  // +1 no violation, -1 violation
                                if (filtered) {
                                    const float4 xf = S.qf[x];
                                    const float t = __fmaf_rn(xf.z, y32[2], __fmaf_rn(xf.y, y32[1], __fmul_rn(xf.x, y32[0])));
                                    const float d = __fmaf_rn(-2.0f, t, xf.w);
                                    if (d > E32) decided = 1;
                                    else if (d < -E32) decided = -1;
                                    if (decided) lc.tri[0]++;
                                }
                                if (!decided) {
                                    if (!have64) make64();
                                    const int4 xq = S.q[x];
                                    const double t = fma((double)xq.z, y64[2], fma((double)xq.y, y64[1], (double)xq.x * y64[0]));
                                    const double d = fma(-2.0, t, (double)xq.w);
                                    if (d > E64) decided = 1;
                                    else if (d < -E64) decided = -1;
                                    if (decided) lc.tri[1]++;
                                }
                                if (!decided) {
                                    lc.tri[2]++;
                                    const int4 xq = S.q[x];
                                    const long long gx1 = (long long)q1.x * xq.x + (long long)q1.y * xq.y + (long long)q1.z * xq.z;
                                    const long long gx2 = (long long)q2.x * xq.x + (long long)q2.y * xq.y + (long long)q2.z * xq.z;
                                    const i128 v = mul64x64(xq.w, detG) - (mul64x64(n1, gx1) + mul64x64(n2, gx2));
                                    if (v < 0) decided = -1;
                                    else if (v > 0) decided = 1;
                                    else {
                                        const long long c1 = g22 * gx1 - g12 * gx2, c2 = g11 * gx2 - g12 * gx1;
                                        const long long coef[3] = {detG - c1 - c2, c1, c2};
                                        const int g[3] = {gi, S.gid[pp], S.gid[kk]};
                                        decided = sos_violates(3, g, coef, S.gid[x]) ? -1 : 1;
                                    }
                                }
                                violated = decided < 0;
                            }
                        }
                        pass = !violated;
                    }
                }
                if (pc.keep_candidates)
                    append_direct(in_sigma, make_int4(i, valid ? S.idx[pp] : 0, valid ? S.idx[kk] : 0, 0), A.cand2,
                                  &cnt->n_cand_out[2], A.cap_cand[2], &cnt->err);
                stage_push(lane, pass, make_int4(i, valid ? S.idx[pp] : 0, valid ? S.idx[kk] : 0, 0), S.st_tri, &S.n_tri,
                           A.tri_out, &cnt->n_tri_pass, A.cap_tri, &cnt->err, DERR_OVF_TRI);
            });
        }
        __syncwarp();

        // ---- phase D: tetrahedra (i,p,k,l): AC3 exact, then AC2 --------------
        for (int r0 = 0; r0 < n_up; r0 += 32) {
            const bool rowok = r0 + lane < n_up;
            const int p = rowok ? S.uplist[r0 + lane] : 0;
            unsigned mask[WORDS];
#pragma unroll
            for (int w = 0; w < WORDS; w++) mask[w] = rowok ? S.Trow[p][w] : 0u;
            warp_expand<WORDS>(lane, mask, p, [&](bool valid1, int pp, int kk) {
                unsigned m2[WORDS];
#pragma unroll
                for (int w = 0; w < WORDS; w++) m2[w] = valid1 ? (S.Trow[pp][w] & S.Trow[kk][w]) : 0u;
                const int tag = valid1 ? (pp | (kk << 8)) : 0;
                warp_expand<WORDS>(lane, m2, tag, [&](bool valid, int pk, int ll) {
                    bool in_sigma = false, pass = false;
                    const int p3 = pk & 255, k3 = pk >> 8;
                    if (valid) {
                        const int4 q1 = S.q[p3], q2 = S.q[k3], q3 = S.q[ll];
                        // cross products (exact in 32 bits: |q| <= 2^13 per axis)
                        const int C1x = q2.y * q3.z - q2.z * q3.y, C1y = q2.z * q3.x - q2.x * q3.z,
                                  C1z = q2.x * q3.y - q2.y * q3.x;
                        const int C2x = q3.y * q1.z - q3.z * q1.y, C2y = q3.z * q1.x - q3.x * q1.z,
                                  C2z = q3.x * q1.y - q3.y * q1.x;
                        const int C3x = q1.y * q2.z - q1.z * q2.y, C3y = q1.z * q2.x - q1.x * q2.z,
                                  C3z = q1.x * q2.y - q1.y * q2.x;
                        const long long D = (long long)q1.x * C1x + (long long)q1.y * C1y + (long long)q1.z * C1z;
                        lc.ac3[3]++;
                        long long N[3] = {0, 0, 0};
                        if (D != 0) {
                            N[0] = (long long)q1.w * C1x + (long long)q2.w * C2x + (long long)q3.w * C3x;
                            N[1] = (long long)q1.w * C1y + (long long)q2.w * C2y + (long long)q3.w * C3y;
                            N[2] = (long long)q1.w * C1z + (long long)q2.w * C2z + (long long)q3.w * C3z;
                            const i128 nn = mul64x64(N[0], N[0]) + mul64x64(N[1], N[1]) + mul64x64(N[2], N[2]);
                            in_sigma = nn <= mul64x64(D, D) * (i128)(4 * si);
                        }
                        if (in_sigma) {
                            lc.cand[3]++;
                            const int sD = D > 0 ? 1 : -1;
                            float y32[3] = {0.f, 0.f, 0.f};
                            double y64[3] = {0.0, 0.0, 0.0};
                            bool have64 = false;
                            if (filtered) {
                                const float rd = __frcp_rn(2.0f * __ll2float_rn(D));
#pragma unroll
                                for (int c = 0; c < 3; c++) y32[c] = __fmul_rn(__ll2float_rn(N[c]), rd);
                            }
                            auto make64 = [&]() {
                                const double rd = 1.0 / (2.0 * (double)D);
                                for (int c = 0; c < 3; c++) y64[c] = (double)N[c] * rd;
                                have64 = true;
                            };
                            if (!filtered) make64();
                            bool violated = false;
#pragma unroll
                            for (int w = 0; w < WORDS; w++) {
                                unsigned b = S.Mrow[p3][w] & S.Mrow[k3][w] & S.Mrow[ll][w];
                                while (b && !violated) {
                                    const int x = 32 * w + __ffs(b) - 1;
                                    b &= b - 1;
                                    int decided = 0;
                                    if (filtered) {
                                        const float4 xf = S.qf[x];
                                        const float t = __fmaf_rn(xf.z, y32[2], __fmaf_rn(xf.y, y32[1], __fmul_rn(xf.x, y32[0])));
                                        const float d = __fmaf_rn(-2.0f, t, xf.w);
                                        if (d > A.tet_eps32) decided = 1;
                                        else if (d < -A.tet_eps32) decided = -1;
                                        if (decided) lc.tet[0]++;
                                    }
                                    if (!decided) {
                                        if (!have64) make64();
                                        const int4 xq = S.q[x];
                                        const double t = fma((double)xq.z, y64[2], fma((double)xq.y, y64[1], (double)xq.x * y64[0]));
                                        const double d = fma(-2.0, t, (double)xq.w);
                                        if (d > A.tet_eps64) decided = 1;
                                        else if (d < -A.tet_eps64) decided = -1;
                                        if (decided) lc.tet[1]++;
                                    }
                                    if (!decided) {
                                        lc.tet[2]++;
                                        const int4 xq = S.q[x];
                                        const i128 qN = mul64x64(xq.x, N[0]) + mul64x64(xq.y, N[1]) + mul64x64(xq.z, N[2]);
                                        i128 v = mul64x64(xq.w, D) - qN;
                                        if (sD < 0) v = -v;
                                        if (v < 0) decided = -1;
                                        else if (v > 0) decided = 1;
                                        else {
                                            const long long D1 = (long long)xq.x * C1x + (long long)xq.y * C1y + (long long)xq.z * C1z;
                                            const long long D2 = (long long)xq.x * C2x + (long long)xq.y * C2y + (long long)xq.z * C2z;
                                            const long long D3 = (long long)xq.x * C3x + (long long)xq.y * C3y + (long long)xq.z * C3z;
                                            const long long coef[4] = {sD * (D - D1 - D2 - D3), sD * D1, sD * D2, sD * D3};
                                            const int g[4] = {gi, S.gid[p3], S.gid[k3], S.gid[ll]};
                                            decided = sos_violates(4, g, coef, S.gid[x]) ? -1 : 1;
                                        }
                                    }
                                    violated = decided < 0;
                                }
                            }
                            pass = !violated;
                        }
                    }
                    const int4 item = make_int4(i, valid ? S.idx[p3] : 0, valid ? S.idx[k3] : 0, valid ? S.idx[ll] : 0);
                    if (pc.keep_candidates)
                        append_direct(in_sigma, item, A.cand3, &cnt->n_cand_out[3], A.cap_cand[3], &cnt->err);
                    stage_push(lane, pass, item, S.st_tet, &S.n_tet, A.tet_out, &cnt->n_tet_out, A.cap_tet, &cnt->err,
                               DERR_OVF_TET);
                });
            });
        }
        __syncwarp();

        // ---- phase E: edges (i,p): AC2 at the edge's orthocentre, exact -------
        for (int r0 = 0; r0 < n_up; r0 += 32) {
            const bool ok = r0 + lane < n_up;
            const int p = ok ? S.uplist[r0 + lane] : 0;
            bool pass = false;
            if (ok) {
                const int4 q = S.q[p];
                const long long D = (long long)q.x * q.x + (long long)q.y * q.y + (long long)q.z * q.z;
                const long long a = q.w;
                bool violated = false;
#pragma unroll
                for (int w = 0; w < WORDS; w++) {
                    unsigned b = S.Mrow[p][w];
                    while (b && !violated) {
                        const int x = 32 * w + __ffs(b) - 1;
                        b &= b - 1;
                        const int4 xq = S.q[x];
                        const long long qq = (long long)q.x * xq.x + (long long)q.y * xq.y + (long long)q.z * xq.z;
                        const long long v = (long long)xq.w * D - a * qq;  // |.| < 2^55
                        lc.edge++;
                        if (v < 0) violated = true;
                        else if (v == 0) {
                            const long long coef[2] = {D - qq, qq};
                            const int g[2] = {gi, S.gid[p]};
                            violated = sos_violates(2, g, coef, S.gid[x]);
                        }
                    }
                }
                pass = !violated;
            }
            stage_push(lane, pass, make_int2(i, ok ? S.idx[p] : 0), S.st_edge, &S.n_edge, A.edge_out, &cnt->n_edge_pass,
                       A.cap_edge, &cnt->err, DERR_OVF_EDGE);
        }
        __syncwarp();
    }
    // drain the staging buffers
    stage_flush(lane, S.st_tet, &S.n_tet, A.tet_out, &cnt->n_tet_out, A.cap_tet, &cnt->err, DERR_OVF_TET);
    stage_flush(lane, S.st_tri, &S.n_tri, A.tri_out, &cnt->n_tri_pass, A.cap_tri, &cnt->err, DERR_OVF_TRI);
    stage_flush(lane, S.st_edge, &S.n_edge, A.edge_out, &cnt->n_edge_pass, A.cap_edge, &cnt->err, DERR_OVF_EDGE);
    // counters: warp reduction, one atomic per warp and counter
    auto red = [&](unsigned v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
        return v;
    };
    unsigned vals[3 + 3 + 1 + 4 + 4];
    int t = 0;
    for (int k = 0; k < 3; k++) vals[t++] = red(lc.tet[k]);
    for (int k = 0; k < 3; k++) vals[t++] = red(lc.tri[k]);
    vals[t++] = red(lc.edge);
    for (int k = 0; k < 4; k++) vals[t++] = red(lc.ac3[k]);
    for (int k = 0; k < 4; k++) vals[t++] = red(lc.cand[k]);
    if (lane == 0) {
        t = 0;
        for (int k = 0; k < 3; k++) atomicAdd(&cnt->ac2_tet[k], (unsigned long long)vals[t++]);
        for (int k = 0; k < 3; k++) atomicAdd(&cnt->ac2_tri[k], (unsigned long long)vals[t++]);
        atomicAdd(&cnt->ac2_edge, (unsigned long long)vals[t++]);
        for (int k = 0; k < 4; k++) atomicAdd(&cnt->ac3[k], (unsigned long long)vals[t++]);
        for (int k = 0; k < 4; k++) atomicAdd(&cnt->n_cand[k], (unsigned long long)vals[t++]);
    }
}

// ---------------------------------------------------------------------------

template <int WORDS>
static int launch_local(ac_ctx* c, LocalArgs& a, cudaStream_t s) {
    int warps = c->opt.block_warps > 0 ? c->opt.block_warps : 8;
    if (warps > 8) warps = 8;  // __launch_bounds__(256)
    while (warps > 1 && (size_t)warps * sizeof(WarpSmem<WORDS>) > 200 * 1024) warps--;
    const size_t smem = (size_t)warps * sizeof(WarpSmem<WORDS>);
    AC_CUDA(cudaFuncSetAttribute(k_local<WORDS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    AC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_local<WORDS>, warps * 32, smem));
    AC_CUDA(cudaGetDevice(&dev));
    AC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(AC_ERR_CUDA, "per-atom kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * sms;
    int64_t need = (a.n + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    AC_CUDA(cudaEventRecord(c->ev[8], s));
    k_local<WORDS><<<(unsigned)blocks, warps * 32, smem, s>>>(a);
    AC_LAUNCHED();
    AC_CUDA(cudaEventRecord(c->ev[9], s));
    c->local_launches++;
    return AC_OK;
}

// Threshold constants (see the header comment for the bound).
static void set_thresholds(const PredConst& pc, int64_t wmax, LocalArgs& a) {
    const double h = pc.h_d, H2 = h * h;
    const double Wb = (double)wmax;
    for (int lvl = 0; lvl < 2; lvl++) {
        const double u = lvl == 0 ? ldexp(1.0, -24) : ldexp(1.0, -53);
        const double g3 = 3 * u / (1 - 3 * u);
        const double dy = 4.0001 * u;
        const double safety = 1.0 + 8 * u;
        // tetrahedron: u(4h^2 + Wmax) + 2 g3 (2h)(h)(1 + dy) + 2 (2h) dy h
        const double tet = (u * (4 * H2 + Wb) + 4 * g3 * H2 * (1 + dy) + 4 * dy * H2) * safety;
        // triangle: u(4h^2 + Wmax) + 2 g3 (2h)(h + e) + 2 (2h) e = k0 + k1 e
        const double k0 = (u * (4 * H2 + Wb) + 4 * g3 * H2) * safety;
        const double k1 = (4 * g3 * h + 4 * h) * safety;
        if (lvl == 0) {
            a.tet_eps32 = nextafterf((float)tet, INFINITY);
            a.tri_k0_32 = nextafterf((float)k0, INFINITY);
            a.tri_k1_32 = nextafterf((float)k1, INFINITY);
        } else {
            a.tet_eps64 = nextafter(tet, INFINITY);
            a.tri_k0_64 = nextafter(k0, INFINITY);
            a.tri_k1_64 = nextafter(k1, INFINITY);
        }
    }
}

int run_local(ac_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    DevCounters h;
    AC_TRY(read_counters(c, &h, s));
    const int maxdeg = h.max_degree;
    int words = maxdeg <= 32 ? 1 : maxdeg <= 64 ? 2 : maxdeg <= 128 ? 4 : maxdeg <= 256 ? 8 : 0;
    if (words == 0) {
        char b[128];
        snprintf(b, sizeof(b), "an atom has %d neighbours; the per-atom kernel handles at most 256", maxdeg);
        return fail(AC_ERR_CAPACITY, b);
    }
    size_t nn = (size_t)(n > 0 ? n : 1);
    if (c->cap_tet == 0) {
        c->cap_tet = (int64_t)nn * 12 + 1024;
        c->cap_tri = (int64_t)nn * 16 + 1024;
        c->cap_edge = (int64_t)nn * 12 + 1024;
    }
    if (c->pc.keep_candidates && c->cap_cand[1] == 0) {
        c->cap_cand[1] = (int64_t)nn * 32 + 1024;
        c->cap_cand[2] = (int64_t)nn * 160 + 1024;
        c->cap_cand[3] = (int64_t)nn * 256 + 1024;
    }
    int64_t wmax = 0;
    {
        // max W over atoms = H2 - A
        wmax = c->pc.H2 - c->pc.A;
    }
    for (int attempt = 0; attempt < 4; attempt++) {
        AC_TRY(c->tet_out.reserve((size_t)c->cap_tet * sizeof(int4)));
        AC_TRY(c->tri_pass.reserve((size_t)c->cap_tri * sizeof(int4)));
        AC_TRY(c->edge_pass.reserve((size_t)c->cap_edge * sizeof(int2)));
        AC_TRY(c->vert_pass.reserve(nn));
        if (c->pc.keep_candidates) {
            AC_TRY(c->cand[1].reserve((size_t)c->cap_cand[1] * sizeof(int2)));
            AC_TRY(c->cand[2].reserve((size_t)c->cap_cand[2] * sizeof(int4)));
            AC_TRY(c->cand[3].reserve((size_t)c->cap_cand[3] * sizeof(int4)));
        }
        // zero the per-pass counters (keep max_degree and err)
        DevCounters* dc = c->counters.as<DevCounters>();
        AC_CUDA(cudaMemsetAsync(dc, 0, offsetof(DevCounters, err), s));
        AC_CUDA(cudaMemsetAsync(c->vert_pass.p, 0, nn, s));
        LocalArgs a;
        memset(&a, 0, sizeof(a));
        a.Ps = c->Ps.as<int4>();
        a.order = c->order.as<int32_t>();
        a.nb_off = c->nb_cnt.as<int64_t>();
        a.nb = c->nb.as<int32_t>();
        a.n = n;
        a.pc = c->pc;
        set_thresholds(c->pc, wmax, a);
        a.tet_out = c->tet_out.as<int4>();
        a.cap_tet = c->cap_tet;
        a.tri_out = c->tri_pass.as<int4>();
        a.cap_tri = c->cap_tri;
        a.edge_out = c->edge_pass.as<int2>();
        a.cap_edge = c->cap_edge;
        a.vert_pass = c->vert_pass.as<uint8_t>();
        if (c->pc.keep_candidates) {
            a.cand1 = c->cand[1].as<int2>();
            a.cand2 = c->cand[2].as<int4>();
            a.cand3 = c->cand[3].as<int4>();
            for (int d = 0; d < 4; d++) a.cap_cand[d] = c->cap_cand[d];
        }
        a.cnt = dc;
        if (n > 0) {
            int rc = words == 1 ? launch_local<1>(c, a, s)
                     : words == 2 ? launch_local<2>(c, a, s)
                     : words == 4 ? launch_local<4>(c, a, s)
                                  : launch_local<8>(c, a, s);
            if (rc) return rc;
        }
        AC_TRY(read_counters(c, &h, s));
        if (h.err & DERR_DEGREE) return fail(AC_ERR_CAPACITY, "neighbour list wider than the kernel's masks");
        bool again = false;
        if ((int64_t)h.n_tet_out > c->cap_tet) {
            c->cap_tet = (int64_t)(h.n_tet_out * 5 / 4) + 1024;
            again = true;
        }
        if ((int64_t)h.n_tri_pass > c->cap_tri) {
            c->cap_tri = (int64_t)(h.n_tri_pass * 5 / 4) + 1024;
            again = true;
        }
        if ((int64_t)h.n_edge_pass > c->cap_edge) {
            c->cap_edge = (int64_t)(h.n_edge_pass * 5 / 4) + 1024;
            again = true;
        }
        for (int d = 1; d < 4; d++)
            if (c->pc.keep_candidates && (int64_t)h.n_cand_out[d] > c->cap_cand[d]) {
                c->cap_cand[d] = (int64_t)(h.n_cand_out[d] * 5 / 4) + 1024;
                again = true;
            }
        if (!again) {
            // clear overflow bits that a successful pass may have left from an earlier attempt
            return AC_OK;
        }
        unsigned zero_err = 0;
        AC_CUDA(cudaMemcpyAsync(&dc->err, &zero_err, sizeof(unsigned), cudaMemcpyHostToDevice, s));
    }
    return fail(AC_ERR_CAPACITY, "output lists kept overflowing");
}

}  // namespace ac
