// The per-atom pass: potential simplices (Section 4.3, Step 1 of Section 3.1)
// and their AC2 tests (Section 4.4, Steps 2-5), fused in one kernel, plus the
// kernel that settles the cases its floating-point bounds left open.
//
// Ownership. A simplex is owned by its vertex with the lowest sorted position
// i. One warp handles one owner at a time and works entirely inside L(i), the
// list of i's neighbours (atoms whose grown balls meet i's, ac_grid.cu), held
// in shared memory as offsets q_x = P_x - P_i (exact integers, exact in FP32
// because |q| <= 2h <= 2^13) and a_x = |q_x|^2 - W_x + W_i. Bitmasks over
// positions in L(i) (WORDS 32-bit words, |L(i)| <= 32 * WORDS) carry:
//   up       positions x > i with edge (i,x) in Sigma_ortho^1 (edge AC3 exact)
//   M[p]     positions adjacent to p (grown balls meet), for p in up
//   T[p]     positions k > p with triangle (i,p,k) in Sigma_ortho^2
// Potential triangles are pairs (p,k), k in M[p] & up, k > p; potential
// tetrahedra are (p,k,l) with l in T[p] & T[k]. Monotonicity of OrthoSize
// (Section 4.3) makes this complete. Candidates are enumerated by random
// access: per-row counts, a prefix sum, and candidate j -> row by binary
// search -> vertex as the rank-th set bit, 32 candidates per warp step.
//
// AC2 at the orthocentre c = P_i + y of sigma. Every ball x that violates it
// (ties included) has pi(c, b_x) <= OrthoSize(sigma) <= alpha, so its grown
// ball contains c, as does every vertex's: x is adjacent to all vertices, so
// the candidates are M[p] & M[k] & M[l] (all of L(i) for the vertex i).
//   Delta_x = pi(c, b_x) - pi(c, b_i) = a_x - 2 q_x . y;  AC2 fails iff some
//   Delta_x < 0 (Delta_x = 0 is settled by the symbolic perturbation below).
//
// Bounded floating point. k_local evaluates y and every Delta_x in one
// precision R (FP32 for AC_PRECISION_FILTERED, FP64 for
// AC_PRECISION_PLAIN_FP64) with a rigorous bound e_y on |y~_c - y_c| for every
// component (u = unit roundoff of R, gamma_3 = 3u/(1-3u), H = 2h >= |q| for
// every q in L(i), A_m = 4h^2 + max W >= |a|; bounds use upward rounding):
//   tetrahedron: C_k = q_{k+1} x q_{k+2} by FMA, |C~ - C| <= e_C = 2u(1+u)H^2;
//     D = q_1.C_1, |D~ - D| <= e_D = gamma_3 (H^3 + sqrt3 H e_C) + sqrt3 H e_C;
//     N = sum a_k C_k, |N~_c - N_c| <= e_N = 6.001 u H^2 sum|a~_k|;
//     y = N / (2D), rho = e_D/|D~| <= 1/8, Y = max_c |y~_c|:
//     e_y = (e_N/(2|D~|) + Y (rho + k)) (1+k) / (1 - rho(1+k) - k), k = 1.01 (u +
//     delta_r), delta_r the reciprocal's relative error (FP32: rcp.approx,
//     documented within 1 ulp, taken as 16u; FP64: correctly rounded, u).
//   triangle: Gram entries by FMA, |g~ - g| <= gamma_3 H^2; det = g11 g22 - g12^2,
//     |det~ - det| <= e_det = 15.01 u H^4; n = adj(G) a, |n~ - n| <= 6.01 u H^2
//     (|a~_1| + |a~_2|); mu = n / (2 det) bounded as y above (e_mu); y = mu_1 q_1
//     + mu_2 q_2, e_y = 2.0001 u (|mu~_1| + |mu~_2|) H + 2 H e_mu.
//   edge: D = |q|^2 (|D~ - D| <= gamma_3 H^2), mu = a / (2D), y = mu q.
// AC3 (|y|^2 <= W_i + A, since |y|^2 - W_i is OrthoSize): S~ = fl(|y~|^2),
// |S~ - |y|^2| <= gamma_3 S~ (1 + gamma_3) + e_y (2|y~|_1 + 3 e_y); W_i + A <=
// 2^24 is exact. AC2: |fl(Delta) - Delta| <= u|fl(Delta)|(1+u) + u A_m +
// 2 gamma_3 H |y~| + 2 sqrt3 H e_y, and |y| <= h once AC3 holds, so a test is
// decided when |fl(Delta)| > (K0 + K1 e_y)(1 + 1.01u), K0 = u A_m +
// 2 gamma_3 H h, K1 = 2 sqrt3 H (1 + gamma_3).
// A simplex whose AC3, or whose AC2 with no decided violator, stays open is
// appended to a pending list (an undecided triangle still counts as potential
// for the enumeration of tetrahedra: a superset is harmless there). Two kernels
// settle the pending simplices: k_resolve_prep, one thread per simplex, takes
// the exact AC3 in 128-bit integers and the FP64 orthocentre from the exact
// integer minors (relative error <= 4.0001 u_64 per component of y); then
// k_resolve_scan, a group of lanes per simplex whose AC3 holds, makes every AC2
// test in FP32 and FP64 from that orthocentre and, where both are undecided,
// in exact 128-bit integers. Keeping the exact arithmetic out of k_local keeps
// its register budget small.
// Edge AC3 and the vertex test are exact 64-bit integers in every mode.
//
// Ties (Section 2, symbolic perturbation): squared radii W_k + eps_k with eps_k
// falling steeply in the INPUT index k. Delta_x is affine in the weights; its
// coefficient on W_x is -|D| < 0, on W_v (v a vertex of sigma) it is
// |D| lambda_v(x), lambda the affine coordinates of the projection of x on
// aff(sigma). When Delta_x = 0 the coefficient of the smallest input index with
// a non-zero coefficient gives the sign:
//   tetrahedron: D lambda_k = det(Q with row k replaced by q_x) = q_x . C_k
//   triangle:    detG lambda = adj(G) (q_1.q_x, q_2.q_x)
//   edge:        D lambda_1 = q.q_x
// and lambda_i = 1 - sum of the others (exact 64-bit integers).
#include <math.h>

#include <type_traits>

#include "ac_internal.cuh"

namespace ac {

constexpr unsigned FULL = 0xffffffffu;
constexpr int STAGE = 32;
constexpr int PAIR_CHUNK = 128;
constexpr int CAND_CAP = 256;  // triangle or tetrahedron candidates written out per batch
constexpr int PL_CAP = 256;    // Sigma^2 pairs listed during the triangle phase

template <int WORDS>
struct WarpSmem {
    static constexpr int M = 32 * WORDS;
    // row positions take 8 bits up to 256 neighbours, 10 bits beyond
    static constexpr int SH = WORDS > 8 ? 10 : 8;
    static constexpr unsigned PM = (1u << SH) - 1u;
    using Pos = typename std::conditional<(WORDS > 8), unsigned short, unsigned char>::type;
    using Pair = typename std::conditional<(WORDS > 8), unsigned, unsigned short>::type;
    float4 qf[M];   // (qx, qy, qz, a_x): coordinates exact, a_x rounded once
    int ai[M];      // a_x exact
    float rs[M];    // sqrt(W_x + A) rounded up
    int idx[M];     // sorted position
    unsigned Mrow[M][WORDS];
    unsigned Trow[M][WORDS];
    unsigned up[WORDS];
    Pos uplist[M];
    unsigned char upf[M];  // edge (i, x) in Sigma^1, by position
    int n_up;
    int n_tet, n_tri, n_edge;
    int rowpre[M + 1];                // prefix sums of candidate counts per row of up
    int pairpre[PAIR_CHUNK + 1];      // prefix sums of tetrahedron candidates per Sigma^2 pair
    Pair plist[PL_CAP];               // Sigma^2 pairs (p | k << SH) in enumeration order
    int n_pl;                         // pairs found (the list holds them while n_pl <= PL_CAP)
    unsigned cand[CAND_CAP];          // candidate codes (p | k << SH [| l << 2 SH]) of the current batch
    int4 st_tet[STAGE];
    int4 st_tri[STAGE];
    int2 st_edge[STAGE];
};

// Eight warps of 64-bit rows must fit four blocks per SM (228 KB, 1 KB reserved per block).
static_assert(sizeof(WarpSmem<2>) * 8 <= 56 * 1024, "narrow per-atom kernel: 4 blocks of 8 warps per SM");

// Constants of the bounds for one precision (derivation in the header comment).
template <class R>
struct Bounds {
    R H, K0, K1, eC, eD_tet, cN, eG, eDet, cn;
    R k2;   // >= 1.01 (u + delta_r): a reciprocal then a product (delta_r: 16u FP32, u FP64)
    R ky;   // 2.0001 u
    R ke;   // 1.0001 u
    R u;
    R g3s;    // gamma_3 (1 + gamma_3)
    R up1;    // >= 1 + 1.01 u
    R two_up; // >= 2 / (1 - delta_r): 1/|X~| <= |rcp(2 X~)| two_up
};

struct LocalArgs {
    const int4* Ps;
    const int32_t* order;
    // L(i): nb[i * nb_stride ..], nb_off[i] entries, when nb_stride > 0;
    // else nb[nb_off[i] .. nb_off[i + 1]]
    const int64_t* nb_off;
    const int32_t* nb;
    int nb_stride;
    int64_t n;
    // Work of one launch: the atoms work[0..n-1], taken through work_next,
    // work_next2 .. work_next5 (counter 0 .. 4: launches running beside one another).
    const int32_t* work;
    int counter;
    // rows of 8 words or more: the per-warp working sets in global memory (one
    // per warp of the launch), where shared memory would hold too few of them;
    // rows of more than 16 words always (they do not fit shared memory)
    void* gws;
    PredConst pc;
    Bounds<float> b32;
    Bounds<double> b64;
    // FP64 thresholds of the resolve kernel (y from exact minors)
    double tet_eps64, tri_k0_64, tri_k1_64;
    int4* tet_out;
    int64_t cap_tet;
    int4* tri_out;
    int64_t cap_tri;
    int2* edge_out;
    int64_t cap_edge;
    uint8_t* vert_pass;
    int4* pending;
    int64_t cap_pending;
    int4* cand3;
    int4* cand2;
    int2* cand1;
    int64_t cap_cand[4];
    DevCounters* cnt;
};

// ---------------------------------------------------------------------------
// directed-rounding arithmetic in one precision

template <class R>
struct Ar;

template <>
struct Ar<float> {
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float mul_up(float a, float b) { return __fmul_ru(a, b); }
    static __device__ __forceinline__ float mul_dn(float a, float b) { return __fmul_rd(a, b); }
    static __device__ __forceinline__ float fma_up(float a, float b, float c) { return __fmaf_ru(a, b, c); }
    static __device__ __forceinline__ float add_up(float a, float b) { return __fadd_ru(a, b); }
    static __device__ __forceinline__ float sub_dn(float a, float b) { return __fsub_rd(a, b); }
    // PTX rcp.approx.ftz.f32 (documented within 1 ulp of 1/a); the bounds
    // below allow a relative error of 16u for it, not a correctly rounded one.
    static __device__ __forceinline__ float rcp(float a) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
    static __device__ __forceinline__ float abs(float a) { return fabsf(a); }
    static __device__ __forceinline__ float max(float a, float b) { return fmaxf(a, b); }
};

template <>
struct Ar<double> {
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double mul_up(double a, double b) { return __dmul_ru(a, b); }
    static __device__ __forceinline__ double mul_dn(double a, double b) { return __dmul_rd(a, b); }
    static __device__ __forceinline__ double fma_up(double a, double b, double c) { return __fma_ru(a, b, c); }
    static __device__ __forceinline__ double add_up(double a, double b) { return __dadd_ru(a, b); }
    static __device__ __forceinline__ double sub_dn(double a, double b) { return __dsub_rd(a, b); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
    static __device__ __forceinline__ double abs(double a) { return fabs(a); }
    static __device__ __forceinline__ double max(double a, double b) { return fmax(a, b); }
};

template <class R>
struct P4 {
    R x, y, z, w;  // offset from P_i and a_x
};

// Position e of L(i) in precision R: FP32 uses the rounded a_x; FP64 takes the
// exact coordinates from FP32 and a_x exactly from the integer copy.
template <class R, int WORDS>
__device__ __forceinline__ P4<R> point(const WarpSmem<WORDS>& S, int e) {
    const float4 v = S.qf[e];
    if (sizeof(R) == 4) return {(R)v.x, (R)v.y, (R)v.z, (R)v.w};
    return {(R)v.x, (R)v.y, (R)v.z, (R)S.ai[e]};
}

// ---------------------------------------------------------------------------
// warp helpers

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

template <class T>
__device__ __forceinline__ void stage_flush(const int lane, T* stage, int* n_stage, T* out, unsigned long long* counter, int64_t cap,
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
__device__ __forceinline__ void append_lanes(unsigned b, bool want, T item, T* out, unsigned long long* counter,
                                          int64_t cap, unsigned* err, unsigned bit) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(b) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(b));
    base = __shfl_sync(FULL, base, leader);
    if (want) {
        unsigned long long slot = base + __popc(b & lanemask_lt());
        if ((int64_t)slot < cap) out[slot] = item;
        else atomicOr(err, bit);
    }
}

// warp-aggregated append of the lanes with want set
template <class T>
__device__ __forceinline__ void append_direct(bool want, const T& item, T* out, unsigned long long* counter, int64_t cap,
                                              unsigned* err, unsigned bit) {
    const unsigned b = __ballot_sync(FULL, want);
    if (b != 0u) append_lanes(b, want, item, out, counter, cap, err, bit);
}

// Staged append: items gather in shared memory and leave in runs of up to
// STAGE (one warp step adds at most 32 = STAGE items).
static_assert(STAGE >= 32, "a warp step must fit the staging buffer");
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

// largest r in [0, n) with pre[r] <= j (pre non-decreasing, pre[0] = 0 <= j)
__device__ __forceinline__ int row_of(const int* pre, int n, int j) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// warp-wide exclusive prefix sum of per-lane counts c; the total goes to *tot
__device__ __forceinline__ int warp_excl(int lane, int c, int* tot) {
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    *tot = __shfl_sync(FULL, incl, 31);
    return incl - c;
}

// bits of word w of a row that lie above position p
__device__ __forceinline__ unsigned above_mask(int w, int p) {
    if (32 * w + 31 <= p) return 0u;
    if (32 * w > p) return FULL;
    return ~((2u << (p & 31)) - 1u);
}

// position of the rank-th set bit of the multi-word mask f(w), w < nw
template <class F>
__device__ __forceinline__ int nth_in_words(int nw, int rank, F&& f) {
    for (int w = 0; w < nw; w++) {
        const unsigned mw = f(w);
        const int pc = __popc(mw);
        if (rank < pc) return 32 * w + nth_set_bit(mw, rank);
        rank -= pc;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// orthocentres with error bounds (see the header comment)

template <class R>
struct Ortho {
    R y0, y1, y2;
    R ey;     // bound on |y~_c - y_c|, every c
    int ac3;  // +1 holds, -1 fails, 0 undecided
};

// AC3 from y~ and its bound: |y|^2 <= T (T exact)
template <class R>
__device__ __forceinline__ int ac3_from(const Ortho<R>& o, R T, const Bounds<R>& B) {
    using A = Ar<R>;
    const R S = A::fma(o.y2, o.y2, A::fma(o.y1, o.y1, A::mul(o.y0, o.y0)));
    const R l1 = A::add_up(A::add_up(A::abs(o.y0), A::abs(o.y1)), A::abs(o.y2));
    const R eS = A::fma_up(o.ey, A::fma_up(R(3), o.ey, A::mul_up(R(2), l1)), A::mul_up(B.g3s, S));
    if (A::sub_dn(S, eS) > T) return -1;
    if (A::add_up(S, eS) < T) return 1;
    return 0;
}

// Bound of a quotient y = N / (2X) computed as fl(N~ r~), r~ = rcp(2 X~) with
// relative error delta_r: e = (eN/(2|X~|) + Y (rho + k)) (1 + k) / (1 - rho (1 + k) - k),
// k >= delta_r + u + delta_r u, rho = e_X/|X~| <= 1/8. No division:
// 1/|X~| <= inv = 2|r~|/(1 - delta_r) and 1/(1 - x) <= 1 + 2x for x <= 1/2.
template <class R>
__device__ __forceinline__ R quotient_bound(R eN, R inv, R Y, R rho, const Bounds<R>& B) {
    using A = Ar<R>;
    const R k = B.k2;
    const R num = A::mul_up(A::fma_up(Y, A::add_up(rho, k), A::mul_up(eN, R(0.5) * inv)), R(1) + k);
    const R x = A::fma_up(rho, R(1) + k, k);
    return A::mul_up(num, A::fma_up(R(2), x, R(1)));
}

template <class R>
__device__ __forceinline__ R cross_c(R bs, R et, R bt, R es) {
    return Ar<R>::fma(bs, et, -Ar<R>::mul(bt, es));
}

template <class R>
__device__ __forceinline__ Ortho<R> ortho_tet(const P4<R>& q1, const P4<R>& q2, const P4<R>& q3, R T,
                                              const Bounds<R>& B) {
    using A = Ar<R>;
    Ortho<R> o;
    // C1 = q2 x q3, C2 = q3 x q1, C3 = q1 x q2
    const R c1x = cross_c(q2.y, q3.z, q2.z, q3.y), c1y = cross_c(q2.z, q3.x, q2.x, q3.z),
            c1z = cross_c(q2.x, q3.y, q2.y, q3.x);
    const R c2x = cross_c(q3.y, q1.z, q3.z, q1.y), c2y = cross_c(q3.z, q1.x, q3.x, q1.z),
            c2z = cross_c(q3.x, q1.y, q3.y, q1.x);
    const R c3x = cross_c(q1.y, q2.z, q1.z, q2.y), c3y = cross_c(q1.z, q2.x, q1.x, q2.z),
            c3z = cross_c(q1.x, q2.y, q1.y, q2.x);
    const R D = A::fma(q1.z, c1z, A::fma(q1.y, c1y, A::mul(q1.x, c1x)));
    const R r = A::rcp(R(2) * D);
    const R inv = A::mul_up(A::abs(r), B.two_up);  // >= 1/|D~|
    const R rho = A::mul_up(B.eD_tet, inv);         // D~ = 0 gives inf: undecided
    if (!(rho <= R(0.125))) {
        o.ac3 = 0;
        o.ey = R(INFINITY);
        o.y0 = o.y1 = o.y2 = R(0);
        return o;
    }
    const R Nx = A::fma(q3.w, c3x, A::fma(q2.w, c2x, A::mul(q1.w, c1x)));
    const R Ny = A::fma(q3.w, c3y, A::fma(q2.w, c2y, A::mul(q1.w, c1y)));
    const R Nz = A::fma(q3.w, c3z, A::fma(q2.w, c2z, A::mul(q1.w, c1z)));
    o.y0 = A::mul(Nx, r);
    o.y1 = A::mul(Ny, r);
    o.y2 = A::mul(Nz, r);
    const R eN = A::mul_up(B.cN, A::add_up(A::add_up(A::abs(q1.w), A::abs(q2.w)), A::abs(q3.w)));
    const R Y = A::max(A::abs(o.y0), A::max(A::abs(o.y1), A::abs(o.y2)));
    o.ey = quotient_bound(eN, inv, Y, rho, B);
    o.ac3 = ac3_from(o, T, B);
    return o;
}

template <class R>
__device__ __forceinline__ Ortho<R> ortho_tri(const P4<R>& q1, const P4<R>& q2, R T, const Bounds<R>& B) {
    using A = Ar<R>;
    Ortho<R> o;
    const R g11 = A::fma(q1.z, q1.z, A::fma(q1.y, q1.y, A::mul(q1.x, q1.x)));
    const R g22 = A::fma(q2.z, q2.z, A::fma(q2.y, q2.y, A::mul(q2.x, q2.x)));
    const R g12 = A::fma(q1.z, q2.z, A::fma(q1.y, q2.y, A::mul(q1.x, q2.x)));
    const R det = A::fma(g11, g22, -A::mul(g12, g12));
    const R r = A::rcp(R(2) * det);
    const R inv = A::mul_up(A::abs(r), B.two_up);  // >= 1/|det~|
    const R rho = A::mul_up(B.eDet, inv);
    if (!(rho <= R(0.125))) {
        o.ac3 = 0;
        o.ey = R(INFINITY);
        o.y0 = o.y1 = o.y2 = R(0);
        return o;
    }
    const R n1 = A::fma(g22, q1.w, -A::mul(g12, q2.w));
    const R n2 = A::fma(g11, q2.w, -A::mul(g12, q1.w));
    const R m1 = A::mul(n1, r), m2 = A::mul(n2, r);
    const R en = A::mul_up(B.cn, A::add_up(A::abs(q1.w), A::abs(q2.w)));
    const R emu = quotient_bound(en, inv, A::max(A::abs(m1), A::abs(m2)), rho, B);
    o.y0 = A::fma(m1, q1.x, A::mul(m2, q2.x));
    o.y1 = A::fma(m1, q1.y, A::mul(m2, q2.y));
    o.y2 = A::fma(m1, q1.z, A::mul(m2, q2.z));
    o.ey = A::mul_up(B.H, A::fma_up(R(2), emu, A::mul_up(B.ky, A::add_up(A::abs(m1), A::abs(m2)))));
    o.ac3 = ac3_from(o, T, B);
    return o;
}

template <class R>
__device__ __forceinline__ Ortho<R> ortho_edge(const P4<R>& q1, const Bounds<R>& B) {
    using A = Ar<R>;
    Ortho<R> o;
    const R D = A::fma(q1.z, q1.z, A::fma(q1.y, q1.y, A::mul(q1.x, q1.x)));
    const R r = A::rcp(R(2) * D);
    const R inv = A::mul_up(r, B.two_up);  // >= 1/D~
    const R rho = A::mul_up(B.eG, inv);    // eG = gamma_3 H^2 bounds |D~ - D|
    const R m = A::mul(q1.w, r);
    const R emu = quotient_bound(A::mul_up(B.u, A::abs(q1.w)), inv, A::abs(m), rho, B);
    o.y0 = A::mul(m, q1.x);
    o.y1 = A::mul(m, q1.y);
    o.y2 = A::mul(m, q1.z);
    o.ey = A::mul_up(B.H, A::fma_up(B.ke, A::abs(m), emu));
    o.ac3 = 1;  // edge AC3 is decided exactly in phase A
    return o;
}

// AC2 scan of one simplex; the candidates of word w are M[p] & M[k] & M[l]
// (nv = 3), M[p] & M[k] (nv = 2) or M[p] (nv = 1). Returns -1 if a candidate
// violates AC2, +1 if every test clears, 0 if none violates but some test is
// undecided at this precision.
template <class R, int WORDS>
__device__ __forceinline__ int ac2_scan(const WarpSmem<WORDS>& S, int nw, const Ortho<R>& o, const Bounds<R>& B, int nv,
                                        int p, int k, int l, unsigned& n_ok) {
    using A = Ar<R>;
    const R E = A::mul_up(A::fma_up(B.K1, o.ey, B.K0), B.up1);  // inf when o.ey is
    bool open = false;
#pragma unroll 1
    for (int w = 0; w < nw; w++) {
        unsigned b = S.Mrow[p][w];
        if (nv >= 2) b &= S.Mrow[k][w];
        if (nv == 3) b &= S.Mrow[l][w];
        while (b) {
            const int x = 32 * w + __ffs(b) - 1;
            b &= b - 1;
            const P4<R> v = point<R>(S, x);
            const R t = A::fma(v.z, o.y2, A::fma(v.y, o.y1, A::mul(v.x, o.y0)));
            const R d = A::fma(R(-2), t, v.w);
            n_ok++;
            if (d < -E) return -1;
            if (!(d > E)) open = true;
        }
    }
    return open ? 0 : 1;
}

// ---------------------------------------------------------------------------

template <int WORDS, class R, bool KEEP>
__global__ void __launch_bounds__(256, 4) k_local(LocalArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using SM = WarpSmem<WORDS>;
    constexpr int MAXM = SM::M;
    constexpr bool is32 = sizeof(R) == 4;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    // working set: shared memory, or (rows of 8 words or more when the launch
    // provides them, always beyond 16 words) one per warp in global memory
    constexpr bool may_global = WORDS >= 8;
    SM& S = (WORDS > 16 || (may_global && A.gws))
                ? reinterpret_cast<SM*>(A.gws)[(size_t)blockIdx.x * (blockDim.x >> 5) + wib]
                : reinterpret_cast<SM*>(smem_raw)[wib];
    DevCounters* cnt = A.cnt;
    const long long Aq = A.pc.A;
    constexpr bool keep = KEEP;  // A.pc.keep_candidates
    const Bounds<R>& B = *reinterpret_cast<const Bounds<R>*>(is32 ? (const void*)&A.b32 : (const void*)&A.b64);
    unsigned n_tet = 0, n_tri = 0, n_edge = 0, n_ac3e = 0, n_ac3t = 0, n_ac3k = 0, n_s1 = 0, n_s2 = 0, n_s3 = 0;
    if (lane == 0) {
        S.n_tet = 0;
        S.n_tri = 0;
        S.n_edge = 0;
    }
    __syncwarp();

    const long long n_items = A.n;
    unsigned long long* next = A.counter == 4   ? &cnt->work_next5
                               : A.counter == 3 ? &cnt->work_next4
                               : A.counter == 2 ? &cnt->work_next3
                               : A.counter == 1 ? &cnt->work_next2
                                                : &cnt->work_next;
    for (;;) {
        long long i_ll = 0;
        if (lane == 0) i_ll = (long long)atomicAdd(next, 1ull);
        i_ll = __shfl_sync(FULL, i_ll, 0);
        if (i_ll >= n_items) break;
        const int i = A.work[i_ll];
        const int4 Pi = A.Ps[i];
        const int Wi = Pi.w;
        const long long si = (long long)Wi + Aq;
        const int gi = A.order[i];
        const int64_t off = A.nb_stride ? (int64_t)i * A.nb_stride : A.nb_off[i];
        const int m = (int)(A.nb_stride ? A.nb_off[i] : A.nb_off[i + 1] - off);
        if (si < 0) {
            if (lane == 0) A.vert_pass[i] = 0;
            continue;
        }
        if (m > MAXM || (A.nb_stride && m > A.nb_stride)) {
            if (lane == 0) atomicOr(&cnt->err, DERR_DEGREE);
            continue;
        }
        const int nw = (m + 31) >> 5;
        const R T = (R)si;  // W_i + A <= 2^24: exact

        // ---- phase A: load L(i) in order of distance from p_i; vertex AC2
        // (Step 5); upper edges with exact edge AC3. The order only changes
        // the order of the AC2 tests: the nearest balls are the likeliest
        // violators of the simplices around p_i, so scans stop sooner.
#pragma unroll 1
        for (int w = 0; w < nw; w++) {
            const int e = 32 * w + lane;
            if (e < m) {
                const int x = A.nb[off + e];
                const int4 o = A.Ps[x];
                const int qx = o.x - Pi.x, qy = o.y - Pi.y, qz = o.z - Pi.z;
                S.idx[e] = x;
                const int D = qx * qx + qy * qy + qz * qz;  // in (0, 2^26]
                // narrow rows: one 32-bit key D * 64 + e, unique (D = 2^26 wraps to e, below every other key)
                S.ai[e] = WORDS <= 2 ? (int)((unsigned)D * 64u + (unsigned)e) : D;
            }
        }
        __syncwarp();
        int xr[WORDS], rr[WORDS];
#pragma unroll
        for (int w = 0; w < WORDS; w++) {
            const int e = 32 * w + lane;
            xr[w] = -1;
            rr[w] = 0;
            if (w < nw && e < m) {
                const int De = S.ai[e];
                int rank = 0;
                if constexpr (WORDS <= 2) {
#pragma unroll 4
                    for (int f = 0; f < m; f++) rank += (unsigned)S.ai[f] < (unsigned)De ? 1 : 0;
                } else {
#pragma unroll 4
                    for (int f = 0; f < m; f++) {
                        const int Df = S.ai[f];
                        rank += (Df < De || (Df == De && f < e)) ? 1 : 0;
                    }
                }
                xr[w] = S.idx[e];
                rr[w] = rank;
            }
        }
        __syncwarp();
        unsigned vert_bad = 0;
#pragma unroll
        for (int w = 0; w < WORDS; w++) {
            if (xr[w] >= 0) {
                const int x = xr[w], e = rr[w];
                const int4 o = A.Ps[x];
                const int qx = o.x - Pi.x, qy = o.y - Pi.y, qz = o.z - Pi.z;
                const int D = qx * qx + qy * qy + qz * qz;  // <= 2^26
                const int ax = D - o.w + Wi;
                S.qf[e] = make_float4((float)qx, (float)qy, (float)qz, (float)ax);
                S.ai[e] = ax;
                S.rs[e] = __fsqrt_ru((float)((long long)o.w + Aq));  // W + A <= 2^24: exact in FP32
                const int gx = A.order[x];
                S.idx[e] = x;
                // Delta_x = a_x at p_i; a tie goes against the larger input index
                if (ax < 0 || (ax == 0 && gx < gi)) vert_bad = 1;
                bool upper = false;
                if (x > i) {
                    // edge AC3: (D + W_i - W_x)^2 <= 4 D (W_i + A)
                    const long long a = (long long)D + Wi - o.w;
                    upper = a * a <= 4ll * D * si;
                    n_ac3e++;
                }
                S.upf[e] = upper ? 1 : 0;
            }
        }
        __syncwarp();
#pragma unroll 1
        for (int w = 0; w < nw; w++) {
            const int e = 32 * w + lane;
            const unsigned b = __ballot_sync(FULL, e < m && S.upf[e] != 0);
            if (lane == 0) S.up[w] = b;
        }
        if (lane == 0)
            for (int w = nw; w < WORDS; w++) S.up[w] = 0u;
        vert_bad = __any_sync(FULL, vert_bad);
        if (lane == 0) A.vert_pass[i] = vert_bad ? 0 : 1;
        __syncwarp();
        {
            int base = 0;
#pragma unroll 1
            for (int w = 0; w < nw; w++) {
                const unsigned b = S.up[w];
                if ((b >> lane) & 1u) S.uplist[base + __popc(b & lanemask_lt())] = (typename SM::Pos)(32 * w + lane);
                base += __popc(b);
            }
            if (lane == 0) {
                S.n_up = base;
                n_s1 += base;
            }
        }
        __syncwarp();
        const int n_up = S.n_up;
        if (keep) {
            for (int r0 = 0; r0 < n_up; r0 += 32) {
                const bool ok = r0 + lane < n_up;
                const int p = ok ? S.uplist[r0 + lane] : 0;
                append_direct(ok, make_int2(i, ok ? S.idx[p] : 0), A.cand1, &cnt->n_cand_out[1], A.cap_cand[1], &cnt->err,
                              DERR_OVF_CAND);
            }
        }

        // ---- phase B: adjacency rows M[p] for p in up ------------------------
        // The rows only filter candidates, so they may hold more than the exact
        // relation: |q_e - q_p|^2 rounded down <= (sqrt s_p + sqrt s_e)^2 rounded up
        // keeps every pair whose grown balls meet (and a few more at the margin).
        if constexpr (WORDS <= 2) {
            // each lane keeps its columns in registers across the rows
            float cx[WORDS], cy[WORDS], cz[WORDS], cr[WORDS];
            bool cv[WORDS];
#pragma unroll
            for (int w = 0; w < WORDS; w++) {
                const int e = 32 * w + lane;
                cv[w] = w < nw && e < m;
                const float4 qe = S.qf[cv[w] ? e : 0];
                cx[w] = qe.x;
                cy[w] = qe.y;
                cz[w] = qe.z;
                cr[w] = S.rs[cv[w] ? e : 0];
            }
#pragma unroll 1
            for (int r = 0; r < n_up; r++) {
                const int p = S.uplist[r];
                const float4 qp = S.qf[p];
                const float rp = S.rs[p];
#pragma unroll
                for (int w = 0; w < WORDS; w++) {
                    const float dx = cx[w] - qp.x, dy = cy[w] - qp.y, dz = cz[w] - qp.z;  // exact: |.| <= 2^14
                    const float d2 = __fmaf_rd(dz, dz, __fmaf_rd(dy, dy, __fmul_rd(dx, dx)));
                    const float rr = __fadd_ru(rp, cr[w]);
                    const bool adj = cv[w] && 32 * w + lane != p && d2 <= __fmul_ru(rr, rr);
                    const unsigned b = __ballot_sync(FULL, adj);  // words past nw come out empty
                    if (lane == 0) {
                        S.Mrow[p][w] = b;
                        S.Trow[p][w] = 0u;
                    }
                }
            }
        } else {
#pragma unroll 1
        for (int r = 0; r < n_up; r++) {
            const int p = S.uplist[r];
            const float4 qp = S.qf[p];
            const float rp = S.rs[p];
#pragma unroll 1
            for (int w = 0; w < nw; w++) {
                const int e = 32 * w + lane;
                bool adj = false;
                if (e < m && e != p) {
                    const float4 qe = S.qf[e];
                    const float dx = qe.x - qp.x, dy = qe.y - qp.y, dz = qe.z - qp.z;  // exact: |.| <= 2^14
                    const float d2 = __fmaf_rd(dz, dz, __fmaf_rd(dy, dy, __fmul_rd(dx, dx)));
                    const float rr = __fadd_ru(rp, S.rs[e]);
                    adj = d2 <= __fmul_ru(rr, rr);
                }
                const unsigned b = __ballot_sync(FULL, adj);
                if (lane == 0) {
                    S.Mrow[p][w] = b;
                    S.Trow[p][w] = 0u;
                }
            }
            if (lane == 0)
                for (int w = nw; w < WORDS; w++) {
                    S.Mrow[p][w] = 0u;
                    S.Trow[p][w] = 0u;
                }
        }
        }
        __syncwarp();

        if (lane == 0) S.n_pl = 0;
        __syncwarp();
        // ---- phase C: triangles (i,p,k): AC3, then AC2 at the orthocentre -----
        // Candidates of row r (p = uplist[r]): k in M[p] & up, k > p. Rows are
        // taken 32 at a time, one per lane; each writes its candidates as codes
        // p | k << SH to cand[] in row order (CAND_CAP per batch), and windows
        // of 32 candidates read them back.
#pragma unroll 1
        for (int r0 = 0; r0 < n_up; r0 += 32) {
            const bool rv = r0 + lane < n_up;
            const int p = rv ? S.uplist[r0 + lane] : 0;
            int c = 0;
            if (rv)
                for (int w = 0; w < nw; w++) c += __popc(S.Mrow[p][w] & S.up[w] & above_mask(w, p));
            int tot;
            const int ex = warp_excl(lane, c, &tot);
#pragma unroll 1
            for (int done = 0; done < tot; done += CAND_CAP) {
                if (c > 0 && ex < done + CAND_CAP && ex + c > done) {
                    int t = ex;
                    for (int w = 0; w < nw; w++) {
                        unsigned b = S.Mrow[p][w] & S.up[w] & above_mask(w, p);
                        while (b) {
                            const int k = 32 * w + __ffs(b) - 1;
                            b &= b - 1;
                            if (t >= done && t < done + CAND_CAP) S.cand[t - done] = (unsigned)p | ((unsigned)k << SM::SH);
                            t++;
                        }
                    }
                }
                __syncwarp();
                const int nbatch = min(CAND_CAP, tot - done);
#pragma unroll 1
                for (int base = 0; base < nbatch; base += 32) {
                    const int j = base + lane;
                    const bool valid = j < nbatch;
                    bool pass = false, pend = false, keep_it = false;
                    int pend_ac3 = 0;
                    int pp = 0, kk = 0;
                    Ortho<R> o;
                    o.ac3 = -1;
                    if (valid) {
                        const unsigned code = S.cand[j];
                        pp = code & SM::PM;
                        kk = code >> SM::SH;
                        n_ac3t++;
                        o = ortho_tri<R>(point<R>(S, pp), point<R>(S, kk), T, B);
                        if (o.ac3 >= 0) {
                            // potential, or not yet excluded: tetrahedra may build on it
                            atomicOr(&S.Trow[pp][kk >> 5], 1u << (kk & 31));
                            if (o.ac3 > 0) {
                                n_s2++;
                                keep_it = true;
                            } else {
                                pend = true;
                                pend_ac3 = 1;
                            }
                        }
                    }
                    {
                        const int r2 = keep_it ? ac2_scan<R>(S, nw, o, B, 2, pp, kk, 0, n_tri) : 1;
                        if (keep_it) {
                            pass = r2 > 0;
                            pend = r2 == 0;
                        }
                    }
                    {
                        // list the pair for the tetrahedron phase (the triangle is potential or undecided)
                        const bool tp = valid && (keep_it || pend_ac3);
                        const unsigned bt = __ballot_sync(FULL, tp);
                        const int slot = S.n_pl + __popc(bt & lanemask_lt());
                        if (tp && slot < PL_CAP) S.plist[slot] = (typename SM::Pair)(pp | (kk << SM::SH));
                        __syncwarp();
                        if (lane == 0) S.n_pl += __popc(bt);
                        __syncwarp();
                    }
                    const int4 item = make_int4(i, valid ? S.idx[pp] : 0, valid ? S.idx[kk] : 0, 0);
                    if (keep)
                        append_direct(keep_it, item, A.cand2, &cnt->n_cand_out[2], A.cap_cand[2], &cnt->err,
                                      DERR_OVF_CAND);
                    append_direct(pend, make_int4(pend_ac3 ? ~i : i, item.y, item.z, -1), A.pending, &cnt->n_pending,
                                  A.cap_pending, &cnt->err, DERR_OVF_PEND);
                    stage_push(lane, pass, item, S.st_tri, &S.n_tri, A.tri_out, &cnt->n_tri_pass, A.cap_tri, &cnt->err,
                               DERR_OVF_TRI);
                }
                __syncwarp();
            }
        }
        __syncwarp();

        // ---- phase D: tetrahedra (i,p,k,l): AC3, then AC2 ----------------------
        // Sigma^2 pairs (p,k) come from the list the triangle phase wrote (or,
        // when it overflowed, from the T rows: row r of up holds popc(T[p]) of
        // them, located by a prefix and a binary search). Pairs are taken
        // PAIR_CHUNK at a time with a prefix over their candidate counts
        // popc(T[p] & T[k]); their candidates l are written as codes
        // p | k << SH | l << 2 SH to cand[] (CAND_CAP per batch) and read back by
        // windows of 32.
        const bool use_list = S.n_pl <= PL_CAP;
        if (!use_list) {
            int run = 0;
            for (int r0 = 0; r0 < n_up; r0 += 32) {
                int c = 0;
                if (r0 + lane < n_up) {
                    const int p = S.uplist[r0 + lane];
                    for (int w = 0; w < nw; w++) c += __popc(S.Trow[p][w]);
                }
                int tot;
                const int ex = warp_excl(lane, c, &tot);
                if (r0 + lane < n_up) S.rowpre[r0 + lane] = run + ex;
                run += tot;
            }
            if (lane == 0) S.rowpre[n_up] = run;
        }
        __syncwarp();
        const int n_pairs = use_list ? S.n_pl : S.rowpre[n_up];
        // pair j of the enumeration: from the list, or located in the T rows
        auto pair_code = [&](int j) -> unsigned {
            if (use_list) return S.plist[j];
            const int r = row_of(S.rowpre, n_up, j);
            const int p = S.uplist[r];
            const int k = nth_in_words(nw, j - S.rowpre[r], [&](int w) { return S.Trow[p][w]; });
            return (unsigned)(p | (k << SM::SH));
        };
        // AC3 then AC2 for the batch of candidate codes in cand[0, nbatch), 32 per window
        auto tet_windows = [&](int nbatch) {
#pragma unroll 1
            for (int base = 0; base < nbatch; base += 32) {
                const int j = base + lane;
                const bool valid = j < nbatch;
                bool pass = false, pend = false, keep_it = false;
                int pend_ac3 = 0;
                int p3 = 0, k3 = 0, ll = 0;
                Ortho<R> o;
                o.ac3 = -1;
                if (valid) {
                    const unsigned code = S.cand[j];
                    p3 = code & SM::PM;
                    k3 = (code >> SM::SH) & SM::PM;
                    ll = code >> (2 * SM::SH);
                    n_ac3k++;
                    o = ortho_tet<R>(point<R>(S, p3), point<R>(S, k3), point<R>(S, ll), T, B);
                    if (o.ac3 > 0) {
                        n_s3++;
                        keep_it = true;
                    } else if (o.ac3 == 0) {
                        pend = true;
                        pend_ac3 = 1;
                    }
                }
                {
                    const int r3 = keep_it ? ac2_scan<R>(S, nw, o, B, 3, p3, k3, ll, n_tet) : 1;
                    if (keep_it) {
                        pass = r3 > 0;
                        pend = r3 == 0;
                    }
                }
                const int4 item = make_int4(i, valid ? S.idx[p3] : 0, valid ? S.idx[k3] : 0, valid ? S.idx[ll] : 0);
                if (keep)
                    append_direct(keep_it, item, A.cand3, &cnt->n_cand_out[3], A.cap_cand[3], &cnt->err,
                                  DERR_OVF_CAND);
                append_direct(pend, make_int4(pend_ac3 ? ~i : i, item.y, item.z, item.w), A.pending, &cnt->n_pending,
                              A.cap_pending, &cnt->err, DERR_OVF_PEND);
                stage_push(lane, pass, item, S.st_tet, &S.n_tet, A.tet_out, &cnt->n_tet_out, A.cap_tet, &cnt->err,
                           DERR_OVF_TET);
            }
            __syncwarp();
        };
        if constexpr (WORDS <= 2) {
            // narrow rows: a lane takes PAIRS_PER_LANE consecutive pairs and keeps their
            // candidate masks T[p] & T[k] in registers; a prefix over the lanes places
            // its candidates in enumeration order
            constexpr int PPL = 2;
#pragma unroll 1
            for (int c0 = 0; c0 < n_pairs; c0 += 32 * PPL) {
                unsigned code[PPL], mk0[PPL], mk1[PPL];
                int mine = 0;
#pragma unroll
                for (int t = 0; t < PPL; t++) {
                    const int j = c0 + PPL * lane + t;
                    code[t] = 0u;
                    mk0[t] = mk1[t] = 0u;
                    if (j < n_pairs) {
                        code[t] = pair_code(j);
                        const int p = code[t] & SM::PM, k = code[t] >> SM::SH;
                        mk0[t] = S.Trow[p][0] & S.Trow[k][0];
                        if (WORDS > 1) mk1[t] = S.Trow[p][WORDS - 1] & S.Trow[k][WORDS - 1];
                        mine += __popc(mk0[t]) + __popc(mk1[t]);
                    }
                }
                int total;
                const int ex = warp_excl(lane, mine, &total);
#pragma unroll 1
                for (int done = 0; done < total; done += CAND_CAP) {
                    if (ex < done + CAND_CAP && ex + mine > done) {
                        int t = ex;
#pragma unroll
                        for (int u = 0; u < PPL; u++) {
#pragma unroll
                            for (int w = 0; w < WORDS; w++) {
                                unsigned b = w == 0 ? mk0[u] : mk1[u];
                                while (b) {
                                    const int l = 32 * w + __ffs(b) - 1;
                                    b &= b - 1;
                                    if (t >= done && t < done + CAND_CAP)
                                        S.cand[t - done] = code[u] | ((unsigned)l << (2 * SM::SH));
                                    t++;
                                }
                            }
                        }
                    }
                    __syncwarp();
                    tet_windows(min(CAND_CAP, total - done));
                }
            }
        } else {
#pragma unroll 1
            for (int c0 = 0; c0 < n_pairs; c0 += PAIR_CHUNK) {
                const int cn = min(PAIR_CHUNK, n_pairs - c0);
                {
                    int run = 0;
                    for (int q0 = 0; q0 < cn; q0 += 32) {
                        int c = 0;
                        if (q0 + lane < cn) {
                            const unsigned code = pair_code(c0 + q0 + lane);
                            const int p = code & SM::PM, k = code >> SM::SH;
                            if (!use_list) S.plist[q0 + lane] = (typename SM::Pair)code;  // chunk-local copy
                            for (int w = 0; w < nw; w++) c += __popc(S.Trow[p][w] & S.Trow[k][w]);
                        }
                        int tot;
                        const int ex = warp_excl(lane, c, &tot);
                        if (q0 + lane < cn) S.pairpre[q0 + lane] = run + ex;
                        run += tot;
                    }
                    if (lane == 0) S.pairpre[cn] = run;
                }
                __syncwarp();
                const int total = S.pairpre[cn];
#pragma unroll 1
                for (int done = 0; done < total; done += CAND_CAP) {
                    for (int q = lane; q < cn; q += 32) {
                        const int a0 = S.pairpre[q], a1 = S.pairpre[q + 1];
                        if (a1 <= done || a0 >= done + CAND_CAP) continue;
                        const unsigned code = S.plist[(use_list ? c0 : 0) + q];
                        const int p = code & SM::PM, k = code >> SM::SH;
                        int t = a0;
                        for (int w = 0; w < nw; w++) {
                            unsigned b = S.Trow[p][w] & S.Trow[k][w];
                            while (b) {
                                const int l = 32 * w + __ffs(b) - 1;
                                b &= b - 1;
                                if (t >= done && t < done + CAND_CAP) S.cand[t - done] = code | ((unsigned)l << (2 * SM::SH));
                                t++;
                            }
                        }
                    }
                    __syncwarp();
                    tet_windows(min(CAND_CAP, total - done));
                }
            }
        }

        // ---- phase E: edges (i,p): AC2 at the edge's orthocentre ---------------
        for (int r0 = 0; r0 < n_up; r0 += 32) {
            const bool ok = r0 + lane < n_up;
            const int p = ok ? S.uplist[r0 + lane] : 0;
            bool pass = false, pend = false;
            Ortho<R> o;
            o.ac3 = -1;
            if (ok) o = ortho_edge<R>(point<R>(S, p), B);
            {
                const int r1 = ok ? ac2_scan<R>(S, nw, o, B, 1, p, 0, 0, n_edge) : 1;
                if (ok) {
                    pass = r1 > 0;
                    pend = r1 == 0;
                }
            }
            const int idp = ok ? S.idx[p] : 0;
            append_direct(pend, make_int4(i, idp, -1, -1), A.pending, &cnt->n_pending, A.cap_pending, &cnt->err,
                          DERR_OVF_PEND);
            stage_push(lane, pass, make_int2(i, idp), S.st_edge, &S.n_edge, A.edge_out, &cnt->n_edge_pass, A.cap_edge,
                       &cnt->err, DERR_OVF_EDGE);
        }
        __syncwarp();
    }
    // drain the staging buffers
    stage_flush(lane, S.st_tet, &S.n_tet, A.tet_out, &cnt->n_tet_out, A.cap_tet, &cnt->err, DERR_OVF_TET);
    stage_flush(lane, S.st_tri, &S.n_tri, A.tri_out, &cnt->n_tri_pass, A.cap_tri, &cnt->err, DERR_OVF_TRI);
    stage_flush(lane, S.st_edge, &S.n_edge, A.edge_out, &cnt->n_edge_pass, A.cap_edge, &cnt->err, DERR_OVF_EDGE);
    // counters: warp reduction, one atomic per warp and counter
    const unsigned vals[9] = {n_tet, n_tri, n_edge, n_ac3e, n_ac3t, n_ac3k, n_s1, n_s2, n_s3};
    unsigned red[9];
#pragma unroll
    for (int t = 0; t < 9; t++) red[t] = __reduce_add_sync(FULL, vals[t]);
    if (lane == 0) {
        const int lvl = is32 ? 0 : 1;
        atomicAdd(&cnt->ac2_tet[lvl], (unsigned long long)red[0]);
        atomicAdd(&cnt->ac2_tri[lvl], (unsigned long long)red[1]);
        atomicAdd(&cnt->ac2_edge, (unsigned long long)red[2]);
        atomicAdd(&cnt->ac3[1], (unsigned long long)red[3]);
        atomicAdd(&cnt->ac3[2], (unsigned long long)red[4]);
        atomicAdd(&cnt->ac3[3], (unsigned long long)red[5]);
        atomicAdd(&cnt->n_cand[1], (unsigned long long)red[6]);
        atomicAdd(&cnt->n_cand[2], (unsigned long long)red[7]);
        atomicAdd(&cnt->n_cand[3], (unsigned long long)red[8]);
    }
}

// ---------------------------------------------------------------------------
// k_resolve_prep / k_resolve_scan: settlement of the pending simplices

__device__ __forceinline__ i128 mul64x64(long long a, long long b) { return (i128)a * (i128)b; }

// The smallest input index among the candidates with a non-zero coefficient
// decides the sign of a Delta that is exactly zero. True if Delta_eps < 0.
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

constexpr int RESOLVE_LANES = 16;

// Exact quantities of an escalated simplex (owner i, vertices v, nv of them),
// relative to p_i: vertex offsets q, a_v = |q_v|^2 - W_v + W_i, grown weights
// s_v = W_v + A, input indices, and the integer minors of its orthocentre
// (y = N / (2 det) for a tetrahedron; mu = (n1, n2) / (2 det) on the Gram
// matrix (g11, g12; g12, g22) for a triangle; mu = a / (2 det) for an edge).
struct Minors {
    long long q[3][3], a[3], sv[3];
    int gv[3];
    long long det, g11, g22, g12, n1, n2, C[3][3], N[3];
};

__device__ __forceinline__ void make_minors(const LocalArgs& A, const int4& Pi, const int* v, int nv, Minors& M) {
    const long long Aq = A.pc.A, Wi = Pi.w;
    for (int t = 0; t < 3; t++) {
        M.q[t][0] = M.q[t][1] = M.q[t][2] = 0;
        M.a[t] = M.sv[t] = 0;
        M.gv[t] = 0;
    }
    for (int t = 0; t < nv; t++) {
        const int4 P = A.Ps[v[t]];
        M.q[t][0] = P.x - Pi.x;
        M.q[t][1] = P.y - Pi.y;
        M.q[t][2] = P.z - Pi.z;
        M.a[t] = M.q[t][0] * M.q[t][0] + M.q[t][1] * M.q[t][1] + M.q[t][2] * M.q[t][2] - P.w + Wi;
        M.sv[t] = (long long)P.w + Aq;
        M.gv[t] = A.order[v[t]];
    }
    M.det = M.g11 = M.g22 = M.g12 = M.n1 = M.n2 = 0;
    for (int t = 0; t < 3; t++) {
        M.N[t] = 0;
        M.C[t][0] = M.C[t][1] = M.C[t][2] = 0;
    }
    const long long(*q)[3] = M.q;
    if (nv == 1) {
        M.det = q[0][0] * q[0][0] + q[0][1] * q[0][1] + q[0][2] * q[0][2];
    } else if (nv == 2) {
        M.g11 = q[0][0] * q[0][0] + q[0][1] * q[0][1] + q[0][2] * q[0][2];
        M.g22 = q[1][0] * q[1][0] + q[1][1] * q[1][1] + q[1][2] * q[1][2];
        M.g12 = q[0][0] * q[1][0] + q[0][1] * q[1][1] + q[0][2] * q[1][2];
        M.det = M.g11 * M.g22 - M.g12 * M.g12;
        M.n1 = M.g22 * M.a[0] - M.g12 * M.a[1];
        M.n2 = M.g11 * M.a[1] - M.g12 * M.a[0];
    } else {
        for (int t = 0; t < 3; t++) {
            const long long* b = q[(t + 1) % 3];
            const long long* e = q[(t + 2) % 3];
            M.C[t][0] = b[1] * e[2] - b[2] * e[1];
            M.C[t][1] = b[2] * e[0] - b[0] * e[2];
            M.C[t][2] = b[0] * e[1] - b[1] * e[0];
        }
        M.det = q[0][0] * M.C[0][0] + q[0][1] * M.C[0][1] + q[0][2] * M.C[0][2];
        for (int c = 0; c < 3; c++) M.N[c] = M.a[0] * M.C[0][c] + M.a[1] * M.C[1][c] + M.a[2] * M.C[2][c];
    }
}

// An escalated simplex whose AC3 holds, with its orthocentre for the AC2
// tests: yf and E32 for the FP32 test (E32 < 0: none), y and E for the FP64 test
// (triangles and tetrahedra; an edge goes to exact integers directly).
struct ResolveScan {
    int i, v0, v1, v2;  // owner and vertices (sorted positions), v1 / v2 = -1 for fewer
    float yf[3];
    float E32;
    double y[3];
    double E;
};
static_assert(sizeof(ResolveScan) == 64, "one scan record per 64 bytes");

// Pending simplex j: exact AC3 where the per-atom kernel left it open, then the
// FP64 orthocentre from the exact minors. False when its AC3 fails.
__device__ __forceinline__ bool prep_item(const LocalArgs& A, int64_t j, ResolveScan& r, unsigned& n_exact,
                                          unsigned (&n_cand)[4]) {
    const int4 rec = A.pending[j];
    const bool ac3_open = rec.x < 0;
    const int i = ac3_open ? ~rec.x : rec.x;
    const int v[3] = {rec.y, rec.z, rec.w};
    const int nv = rec.z < 0 ? 1 : rec.w < 0 ? 2 : 3;
    const int4 Pi = A.Ps[i];
    const long long si = (long long)Pi.w + A.pc.A;
    Minors M;
    make_minors(A, Pi, v, nv, M);
    if (ac3_open) {
        n_exact++;
        bool ok;
        if (nv == 2)
            ok = M.det > 0 && mul64x64(M.n1, M.a[0]) + mul64x64(M.n2, M.a[1]) <= (i128)(4 * M.det) * (i128)si;
        else
            ok = M.det != 0 && mul64x64(M.N[0], M.N[0]) + mul64x64(M.N[1], M.N[1]) + mul64x64(M.N[2], M.N[2]) <=
                                   mul64x64(M.det, M.det) * (i128)(4 * si);
        if (!ok) return false;
        n_cand[nv]++;
        if (A.pc.keep_candidates) {
            const int4 item = make_int4(i, v[0], v[1], nv == 3 ? v[2] : 0);
            const unsigned long long slot = atomicAdd(&A.cnt->n_cand_out[nv], 1ull);
            if ((int64_t)slot < A.cap_cand[nv]) (nv == 3 ? A.cand3 : A.cand2)[slot] = item;
            else atomicOr(&A.cnt->err, DERR_OVF_CAND);
        }
    }
    r.i = i;
    r.v0 = v[0];
    r.v1 = nv >= 2 ? v[1] : -1;
    r.v2 = nv == 3 ? v[2] : -1;
    // FP64 orthocentre from the exact minors and its decision threshold; ey64
    // bounds |y64_c - y_c| for every c
    double y[3] = {0, 0, 0}, E = 0.0, ey64 = 0.0;
    if (nv == 2) {
        const double rd = 1.0 / (2.0 * (double)M.det);
        const double m1 = (double)M.n1 * rd, m2 = (double)M.n2 * rd;
        double e = 0.0;
        for (int c = 0; c < 3; c++) {
            y[c] = fma(m1, (double)M.q[0][c], m2 * (double)M.q[1][c]);
            e += fabs(m1) * fabs((double)M.q[0][c]) + fabs(m2) * fabs((double)M.q[1][c]);
        }
        e *= 6.05 * 1.1102230246251565e-16 * (1.0 + 1e-10);
        ey64 = e;
        E = (A.tri_k0_64 + A.tri_k1_64 * e) * (1.0 + 1e-10);
    } else if (nv == 3) {
        const double rd = 1.0 / (2.0 * (double)M.det);
        for (int c = 0; c < 3; c++) y[c] = (double)M.N[c] * rd;
        ey64 = 4.0002 * 1.1102230246251565e-16 * fmax(fabs(y[0]), fmax(fabs(y[1]), fabs(y[2])));
        E = A.tet_eps64;
    }
    // filtered mode: an FP32 test first, with y rounded to FP32 from y64 and the
    // per-atom kernel's FP32 threshold for |y~_c - y_c| <= ey32, where
    // |y32_c - y_c| <= u32 |y64_c| + ey64 <= 1.0001 u32 |y32_c| + ey64
    r.E32 = -1.0f;
    r.yf[0] = r.yf[1] = r.yf[2] = 0.0f;
    if (A.pc.precision == AC_PRECISION_FILTERED && nv >= 2) {
        double ymax = 0.0;
        for (int c = 0; c < 3; c++) {
            r.yf[c] = __double2float_rn(y[c]);
            ymax = fmax(ymax, fabs((double)r.yf[c]));
        }
        const double ey32 = 1.0001 * 5.9604644775390625e-08 * ymax + ey64;
        const double e32 = ((double)A.b32.K1 * ey32 + (double)A.b32.K0) * (double)A.b32.up1 * (1.0 + 1e-6);
        r.E32 = __double2float_ru(e32);
    }
    for (int c = 0; c < 3; c++) r.y[c] = y[c];
    r.E = E;
    return true;
}

// One thread per pending simplex (the FP64 and 128-bit work at full lane
// occupancy); the simplices whose AC3 holds go to the scan list. n_pending < 0:
// the count the per-atom pass left on the device.
__global__ void __launch_bounds__(128, 4) k_resolve_prep(LocalArgs A, int64_t n_pending, ResolveScan* __restrict__ scan) {
    DevCounters* cnt = A.cnt;
    const int lane = threadIdx.x & 31;
    const int64_t np = n_pending >= 0 ? n_pending
                                      : (int64_t)min(cnt->n_pending, (unsigned long long)A.cap_pending);
    unsigned n_exact = 0, n_cand[4] = {0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps step together, so the append below is warp-aggregated
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); j0 < np; j0 += stride) {
        const int64_t j = j0 + lane;
        ResolveScan r;
        const bool keep = j < np && prep_item(A, j, r, n_exact, n_cand);
        const unsigned b = __ballot_sync(FULL, keep);
        if (!b) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&cnt->n_scan, (unsigned long long)__popc(b));
        base = __shfl_sync(FULL, base, 0);
        if (keep) scan[base + __popc(b & lanemask_lt())] = r;  // at most n_pending <= the list's capacity
    }
    n_exact = __reduce_add_sync(FULL, n_exact);
    n_cand[2] = __reduce_add_sync(FULL, n_cand[2]);
    n_cand[3] = __reduce_add_sync(FULL, n_cand[3]);
    if (lane == 0) {
        if (n_exact) atomicAdd(&cnt->ac3_exact, (unsigned long long)n_exact);
        if (n_cand[2]) atomicAdd(&cnt->n_cand[2], (unsigned long long)n_cand[2]);
        if (n_cand[3]) atomicAdd(&cnt->n_cand[3], (unsigned long long)n_cand[3]);
    }
}

// Exact AC2 decision for candidate x (offset qx from p_i, a_x = ax) against the
// escalated simplex (i, v): the sign of Delta_x times the orthocentre's
// denominator in 128-bit integers, and the symbolic perturbation when it is
// zero. Out of line: the FP32 and FP64 tests settle nearly every case.
__device__ __noinline__ bool exact_violates(const LocalArgs& A, int i, const int* v, int nv, int x,
                                            const long long* qx, long long ax) {
    const int4 Pi = A.Ps[i];
    Minors M;
    make_minors(A, Pi, v, nv, M);
    const long long(*q)[3] = M.q;
    const int gi = A.order[i], gx = A.order[x];
    if (nv == 1) {
        const long long qq = q[0][0] * qx[0] + q[0][1] * qx[1] + q[0][2] * qx[2];
        const long long vv = ax * M.det - M.a[0] * qq;  // |.| < 2^55
        if (vv != 0) return vv < 0;
        const long long coef[2] = {M.det - qq, qq};
        const int g[2] = {gi, M.gv[0]};
        return sos_violates(2, g, coef, gx);
    }
    if (nv == 2) {
        const long long gx1 = q[0][0] * qx[0] + q[0][1] * qx[1] + q[0][2] * qx[2];
        const long long gx2 = q[1][0] * qx[0] + q[1][1] * qx[1] + q[1][2] * qx[2];
        const i128 vv = mul64x64(ax, M.det) - (mul64x64(M.n1, gx1) + mul64x64(M.n2, gx2));
        if (vv != 0) return vv < 0;
        const long long c1 = M.g22 * gx1 - M.g12 * gx2, c2 = M.g11 * gx2 - M.g12 * gx1;
        const long long coef[3] = {M.det - c1 - c2, c1, c2};
        const int g[3] = {gi, M.gv[0], M.gv[1]};
        return sos_violates(3, g, coef, gx);
    }
    const int sD = M.det > 0 ? 1 : -1;
    i128 vv = mul64x64(ax, M.det) - (mul64x64(qx[0], M.N[0]) + mul64x64(qx[1], M.N[1]) + mul64x64(qx[2], M.N[2]));
    if (sD < 0) vv = -vv;
    if (vv != 0) return vv < 0;
    const long long D1 = qx[0] * M.C[0][0] + qx[1] * M.C[0][1] + qx[2] * M.C[0][2];
    const long long D2 = qx[0] * M.C[1][0] + qx[1] * M.C[1][1] + qx[2] * M.C[1][2];
    const long long D3 = qx[0] * M.C[2][0] + qx[1] * M.C[2][1] + qx[2] * M.C[2][2];
    const long long coef[4] = {sD * (M.det - D1 - D2 - D3), sD * D1, sD * D2, sD * D3};
    const int g[4] = {gi, M.gv[0], M.gv[1], M.gv[2]};
    return sos_violates(4, g, coef, gx);
}

__device__ __forceinline__ bool meet(long long D, long long s1, long long s2) {
    const long long t = D - s1 - s2;
    return t <= 0 || t * t <= 4 * s1 * s2;
}

// The AC2 tests of the scan list: RESOLVE_LANES lanes per simplex share the
// entries of L(i), each candidate adjacent to every vertex tested in FP32
// (filtered mode), then FP64, then exact integers; the group stops at the
// first violator. Survivors join the output lists.
__global__ void __launch_bounds__(128) k_resolve_scan(LocalArgs A, const ResolveScan* __restrict__ scan) {
    DevCounters* cnt = A.cnt;
    const int lane = threadIdx.x & 31, sub = lane % RESOLVE_LANES;
    const unsigned gmask = ((1u << RESOLVE_LANES) - 1u) << (lane & ~(RESOLVE_LANES - 1));
    const int64_t ns = (int64_t)min(cnt->n_scan, (unsigned long long)A.cap_pending);
    const long long Aq = A.pc.A;
    unsigned c32[4] = {0, 0, 0, 0}, c64[4] = {0, 0, 0, 0}, cx[4] = {0, 0, 0, 0};  // by vertex count
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / RESOLVE_LANES;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / RESOLVE_LANES; j < ns; j += groups) {
        const ResolveScan r = scan[j];
        const int v[3] = {r.v0, r.v1, r.v2};
        const int nv = r.v1 < 0 ? 1 : r.v2 < 0 ? 2 : 3;
        const int4 Pi = A.Ps[r.i];
        const long long Wi = Pi.w;
        int qv[3][3];  // vertex offsets from p_i: below 2^14 in magnitude
        long long sv[3];
        for (int t = 0; t < 3; t++) {
            const int4 P = A.Ps[t < nv ? v[t] : r.i];
            qv[t][0] = P.x - Pi.x;
            qv[t][1] = P.y - Pi.y;
            qv[t][2] = P.z - Pi.z;
            sv[t] = (long long)P.w + Aq;
        }
        const int64_t off = A.nb_stride ? (int64_t)r.i * A.nb_stride : A.nb_off[r.i];
        const int m = A.nb_stride ? min((int)A.nb_off[r.i], A.nb_stride) : (int)(A.nb_off[r.i + 1] - off);
        bool violated = false;
        for (int e0 = 0; e0 < m; e0 += RESOLVE_LANES) {
            const int e = e0 + sub;
            bool viol = false;
            if (e < m) {
                const int x = A.nb[off + e];
                if (x != v[0] && x != v[1] && x != v[2]) {
                    const int4 Px = A.Ps[x];
                    const long long sx = (long long)Px.w + Aq;
                    const int qx0 = Px.x - Pi.x, qx1 = Px.y - Pi.y, qx2 = Px.z - Pi.z;
                    bool adj = true;
                    for (int t = 0; t < nv && adj; t++) {
                        // both points lie within 2h <= 2^13 quanta of p_i: differences below 2^14
                        const int dx = qx0 - qv[t][0], dy = qx1 - qv[t][1], dz = qx2 - qv[t][2];
                        adj = meet((long long)(dx * dx + dy * dy + dz * dz), sv[t], sx);
                    }
                    if (adj) {
                        const long long ax = (long long)qx0 * qx0 + (long long)qx1 * qx1 + (long long)qx2 * qx2 - Px.w + Wi;
                        int dec = 0;
                        if (r.E32 >= 0.0f) {
                            // the per-atom kernel's FP32 test (same operands and operations)
                            const float t = __fmaf_rn((float)qx2, r.yf[2],
                                                      __fmaf_rn((float)qx1, r.yf[1], __fmul_rn((float)qx0, r.yf[0])));
                            const float d = __fmaf_rn(-2.0f, t, (float)ax);
                            if (d > r.E32) dec = 1;
                            else if (d < -r.E32) dec = -1;
                            if (dec) c32[nv]++;
                        }
                        if (nv >= 2 && !dec) {
                            const double t = fma((double)qx2, r.y[2], fma((double)qx1, r.y[1], (double)qx0 * r.y[0]));
                            const double d = fma(-2.0, t, (double)ax);
                            if (d > r.E) dec = 1;
                            else if (d < -r.E) dec = -1;
                            if (dec) c64[nv]++;
                        }
                        if (!dec) {
                            cx[nv]++;
                            const long long qx[3] = {qx0, qx1, qx2};
                            dec = exact_violates(A, r.i, v, nv, x, qx, ax) ? -1 : 1;
                        }
                        viol = dec < 0;
                    }
                }
            }
            if (__any_sync(gmask, viol)) {
                violated = true;
                break;
            }
        }
        if (violated || sub != 0) continue;
        if (nv == 3) {
            const unsigned long long slot = atomicAdd(&cnt->n_tet_out, 1ull);
            if ((int64_t)slot < A.cap_tet) A.tet_out[slot] = make_int4(r.i, v[0], v[1], v[2]);
            else atomicOr(&cnt->err, DERR_OVF_TET);
        } else if (nv == 2) {
            const unsigned long long slot = atomicAdd(&cnt->n_tri_pass, 1ull);
            if ((int64_t)slot < A.cap_tri) A.tri_out[slot] = make_int4(r.i, v[0], v[1], 0);
            else atomicOr(&cnt->err, DERR_OVF_TRI);
        } else {
            const unsigned long long slot = atomicAdd(&cnt->n_edge_pass, 1ull);
            if ((int64_t)slot < A.cap_edge) A.edge_out[slot] = make_int2(r.i, v[0]);
            else atomicOr(&cnt->err, DERR_OVF_EDGE);
        }
    }
    // counters: one atomic per warp and level
    unsigned red[7] = {c32[3], c64[3], cx[3], c32[2], c64[2], cx[2], cx[1] + c64[1] + c32[1]};
#pragma unroll
    for (int t = 0; t < 7; t++) red[t] = __reduce_add_sync(FULL, red[t]);
    if (lane == 0) {
        for (int k = 0; k < 3; k++) {
            if (red[k]) atomicAdd(&cnt->ac2_tet[k], (unsigned long long)red[k]);
            if (red[3 + k]) atomicAdd(&cnt->ac2_tri[k], (unsigned long long)red[3 + k]);
        }
        if (red[6]) atomicAdd(&cnt->ac2_edge, (unsigned long long)red[6]);
    }
}

// ---------------------------------------------------------------------------

template <int WORDS, class R>
static int launch_local(ac_ctx* c, const LocalArgs& a, int64_t max_items, int warps_req, cudaStream_t s) {
    int warps = warps_req > 0 ? warps_req : c->opt.block_warps > 0 ? c->opt.block_warps : 8;
    if (warps > 8) warps = 8;  // __launch_bounds__(256)
    while (warps > 1 && (size_t)warps * sizeof(WarpSmem<WORDS>) > 200 * 1024) warps--;
    const size_t smem = (size_t)warps * sizeof(WarpSmem<WORDS>);
    void (*kern)(LocalArgs) = a.pc.keep_candidates ? k_local<WORDS, R, true> : k_local<WORDS, R, false>;
    AC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    AC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    AC_CUDA(cudaGetDevice(&dev));
    AC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(AC_ERR_CUDA, "per-atom kernel does not fit on an SM");
    int64_t blocks = (int64_t)per_sm * sms;
    int64_t need = (max_items + warps - 1) / warps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, warps * 32, smem, s>>>(a);
    AC_LAUNCHED();
    c->local_launches++;
    return AC_OK;
}

// Atoms with 513..1024 neighbours: rows of 32 words, each warp's working set
// (about 300 KB) in global memory, one warp per atom up to 16 per SM (the
// kernel waits on memory: warps hide it), 2 GB of working sets at most;
// blocks of two warps.
// A launch whose per-warp working sets live in global memory (rows of 8 words
// or more): as many warps as can be resident (two-warp blocks, 64 registers:
// 32 warps per SM) where shared memory would allow 2 to 8, their working sets
// within 4 GB. The tiers that use it run one after another on one stream and
// share the buffer.
template <int WORDS, class R>
static int launch_global(ac_ctx* c, LocalArgs a, cudaStream_t s) {
    static_assert(WORDS >= 8, "narrow rows keep their working sets in shared memory");
    int dev = 0, sms = 0;
    AC_CUDA(cudaGetDevice(&dev));
    AC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = ((int64_t)4 << 30) / (int64_t)sizeof(WarpSmem<WORDS>);
    const int64_t warps = std::min<int64_t>(std::min<int64_t>(a.n, 32 * (int64_t)sms), cap);
    const int64_t blocks = (warps + 1) / 2;
    AC_TRY(c->huge_ws.reserve((size_t)blocks * 2 * sizeof(WarpSmem<WORDS>), s));
    a.gws = c->huge_ws.p;
    void (*kern)(LocalArgs) = a.pc.keep_candidates ? k_local<WORDS, R, true> : k_local<WORDS, R, false>;
    kern<<<(unsigned)blocks, 64, 0, s>>>(a);
    AC_LAUNCHED();
    c->local_launches++;
    return AC_OK;
}

template <class R>
static int launch_words(ac_ctx* c, int words, const LocalArgs& a, int warps, cudaStream_t s) {
    return words == 1 ? launch_local<1, R>(c, a, a.n, warps, s)
           : words == 2 ? launch_local<2, R>(c, a, a.n, warps, s)
           : words == 4 ? launch_local<4, R>(c, a, a.n, warps, s)
           : words == 8 ? launch_local<8, R>(c, a, a.n, warps, s)
                        : launch_local<16, R>(c, a, a.n, warps, s);
}

// One per-atom pass over the work order (decreasing neighbour count). When
// some atom has more than 64 neighbours, those atoms (the head of the order)
// run on a side stream, concurrently with the narrow kernel (64-bit rows:
// smaller shared-memory footprint, twice the resident warps) over the rest,
// in tiers of the row width they need: more than 512 neighbours (32 words),
// 257..512 (16), 129..256 (8), each with its working sets in global memory at
// 32 warps per SM (shared memory would hold 2 to 8 of them), and 65..128 (4),
// whose working sets stay in shared memory (in global memory that tier ran
// slower on a 100k-atom globule).
template <class R>
static int launch_pass(ac_ctx* c, int words, LocalArgs& a, cudaStream_t s) {
    AC_TRY(stage_mark(c, 8, s));
    const int32_t* work = c->work.as<int32_t>();
    const int64_t n_wide = words > 2 ? c->n_wide : 0;
    const int64_t n_huge = words > 16 ? std::min(c->n_huge, n_wide) : 0;
    const int64_t n_w256 = words > 8 ? std::max(std::min(c->n_w256, n_wide), n_huge) : n_huge;
    const int64_t n_w128 = words > 4 ? std::max(std::min(c->n_w128, n_wide), n_w256) : n_w256;
    if (n_wide > 0) {
        AC_CUDA(cudaEventRecord(c->ev_fork, s));
        AC_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        if (n_huge > 0) {
            LocalArgs huge = a;
            huge.work = work;
            huge.n = n_huge;
            huge.counter = 2;
            AC_TRY((launch_global<32, R>(c, huge, c->side)));
        }
        // [first, last) of the work order in a tier of the given row width
        auto tier = [&](int64_t first, int64_t last, int w, int counter) -> int {
            if (last <= first) return AC_OK;
            LocalArgs t = a;
            t.work = work + first;
            t.n = last - first;
            t.counter = counter;
            return w == 16 ? launch_global<16, R>(c, t, c->side)
                   : w == 8 ? launch_global<8, R>(c, t, c->side)
                            : launch_words<R>(c, w, t, 0, c->side);
        };
        AC_TRY(tier(n_huge, n_w256, 16, 1));
        AC_TRY(tier(n_w256, n_w128, 8, 3));
        AC_TRY(tier(n_w128, n_wide, 4, 4));
        AC_CUDA(cudaEventRecord(c->ev_join, c->side));
    }
    LocalArgs narrow = a;
    narrow.work = work + n_wide;
    narrow.n = a.n - n_wide;
    narrow.counter = 0;
    if (narrow.n > 0) AC_TRY(launch_words<R>(c, n_wide > 0 ? 2 : words, narrow, 0, s));
    if (n_wide > 0) AC_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
    AC_TRY(stage_mark(c, 9, s));
    return AC_OK;
}

// Constants of the bounds at unit roundoff u (derivation in the header comment).
template <class R>
static void set_bounds(double u, double h, int64_t wmax, Bounds<R>& b) {
    // reciprocal error: FP32 rcp.approx is documented within 1 ulp (2u); 16u is
    // taken, a wide margin at no measurable cost. FP64 is correctly rounded (u).
    const double delta_r = sizeof(R) == 4 ? 16.0 * u : u;
    auto up = [](double x) {
        const R r = (R)(x * (1.0 + 1e-12));
        return (double)r >= x ? r : (R)nextafter(r, (R)INFINITY);
    };
    const double H = 2.0 * h, g3 = 3 * u / (1 - 3 * u), s3 = sqrt(3.0) * (1 + 1e-7);
    const double Am = 4 * h * h + (double)wmax;
    const double slack = 1.0 + 64 * u;
    b.H = up(H);
    b.eC = up(2 * u * (1 + u) * H * H * slack);
    const double eC = (double)b.eC;
    b.eD_tet = up((g3 * (H * H * H + s3 * H * eC) + s3 * H * eC) * slack);
    b.cN = up(6.001 * u * H * H * slack);
    b.eG = up(g3 * H * H * slack);
    b.eDet = up(15.01 * u * H * H * H * H * slack);
    b.cn = up(6.01 * u * H * H * slack);
    b.K0 = up((u * Am + 2 * g3 * H * h) * slack);
    b.K1 = up(2 * s3 * H * (1 + g3) * slack);
    b.k2 = up((delta_r + u) * 1.01);
    b.ky = up(2.0001 * u);
    b.ke = up(1.0001 * u);
    b.u = up(u);
    b.g3s = up(g3 * (1 + g3) * slack);
    b.up1 = up(1.0 + 1.01 * u * slack);
    b.two_up = up(2.0 / (1.0 - delta_r) * (1.0 + 4.0 * u));
}

static void set_constants(const PredConst& pc, int64_t wmax, LocalArgs& a) {
    const double h = pc.h_d, H = 2.0 * h;
    set_bounds<float>(ldexp(1.0, -24), h, wmax, a.b32);
    set_bounds<double>(ldexp(1.0, -53), h, wmax, a.b64);
    // resolve kernel: y from exact minors with relative error <= 4.0001 u64 per component
    const double v = ldexp(1.0, -53), g3d = 3 * v / (1 - 3 * v), dy = 4.0001 * v, sf = 1.0 + 16 * v;
    const double s3 = sqrt(3.0) * (1 + 1e-7), Am = 4 * h * h + (double)wmax;
    a.tet_eps64 = nextafter((v * Am + 2 * g3d * H * h * (1 + dy) + 2 * dy * H * h * s3) * sf * (1 + 1e-12), INFINITY);
    a.tri_k0_64 = nextafter((v * Am + 2 * g3d * H * h) * sf * (1 + 1e-12), INFINITY);
    a.tri_k1_64 = nextafter((2 * g3d * H + 2 * H) * s3 * sf * (1 + 1e-12), INFINITY);
}

// blocks of a resolve kernel for up to `items` escalated simplices: `lanes`
// threads per simplex, at most one wave of 16 blocks per SM (the kernels stride
// over the rest, so the cap only bounds the blocks that start with nothing to
// do when a first build sizes the launch by the list's capacity)
static unsigned resolve_blocks(int64_t items, int lanes) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    const int64_t want = (items * lanes + 127) / 128;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
}

int run_local(ac_ctx* c, cudaStream_t s) {
    const int64_t n = c->n;
    DevCounters h = c->replaying ? c->rec.post : c->hc;  // read after the neighbour count pass
    const int maxdeg = h.max_degree;
    int words = maxdeg <= 32 ? 1 : maxdeg <= 64 ? 2 : maxdeg <= 128 ? 4 : maxdeg <= 256 ? 8 : maxdeg <= 512 ? 16
              : maxdeg <= MAX_DEGREE ? 32 : 0;
    if (words == 0) {
        char b[128];
        snprintf(b, sizeof(b), "an atom has %d neighbours; the per-atom kernel handles at most %d", maxdeg, MAX_DEGREE);
        return fail(AC_ERR_CAPACITY, b);
    }
    size_t nn = (size_t)(n > 0 ? n : 1);
    if (c->cap_tet == 0) {
        c->cap_tet = (int64_t)nn * 12 + 1024;
        c->cap_tri = (int64_t)nn * 16 + 1024;
        c->cap_edge = (int64_t)nn * 12 + 1024;
        c->cap_pending = (int64_t)nn * 2 + 4096;  // escalated simplices: about 1.3 per atom with probe radii
    }
    if (c->pc.keep_candidates && c->cap_cand[1] == 0) {
        c->cap_cand[1] = (int64_t)nn * 32 + 1024;
        c->cap_cand[2] = (int64_t)nn * 160 + 1024;
        c->cap_cand[3] = (int64_t)nn * 256 + 1024;
    }
    const int64_t wmax = c->pc.H2 - c->pc.A;  // max W over the atoms
    for (int attempt = 0; attempt < 4; attempt++) {
        AC_TRY(c->tet_out.reserve((size_t)c->cap_tet * sizeof(int4), s));
        AC_TRY(c->tri_pass.reserve((size_t)c->cap_tri * sizeof(int4), s));
        AC_TRY(c->edge_pass.reserve((size_t)c->cap_edge * sizeof(int2), s));
        AC_TRY(c->pending.reserve((size_t)c->cap_pending * sizeof(int4), s));
        AC_TRY(c->resolve_scan.reserve((size_t)c->cap_pending * sizeof(ResolveScan), s));
        ResolveScan* scan = c->resolve_scan.as<ResolveScan>();
        AC_TRY(c->vert_pass.reserve(nn, s));
        if (c->pc.keep_candidates) {
            AC_TRY(c->cand[1].reserve((size_t)c->cap_cand[1] * sizeof(int2), s));
            AC_TRY(c->cand[2].reserve((size_t)c->cap_cand[2] * sizeof(int4), s));
            AC_TRY(c->cand[3].reserve((size_t)c->cap_cand[3] * sizeof(int4), s));
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
        a.nb_stride = c->nb_stride;
        a.n = n;
        a.pc = c->pc;
        set_constants(c->pc, wmax, a);
        a.tet_out = c->tet_out.as<int4>();
        a.cap_tet = c->cap_tet;
        a.tri_out = c->tri_pass.as<int4>();
        a.cap_tri = c->cap_tri;
        a.edge_out = c->edge_pass.as<int2>();
        a.cap_edge = c->cap_edge;
        a.vert_pass = c->vert_pass.as<uint8_t>();
        a.pending = c->pending.as<int4>();
        a.cap_pending = c->cap_pending;
        if (c->pc.keep_candidates) {
            a.cand1 = c->cand[1].as<int2>();
            a.cand2 = c->cand[2].as<int4>();
            a.cand3 = c->cand[3].as<int4>();
            for (int d = 0; d < 4; d++) a.cap_cand[d] = c->cap_cand[d];
        }
        a.cnt = dc;
        if (n > 0) {
            const int rc = c->pc.precision == AC_PRECISION_FILTERED ? launch_pass<float>(c, words, a, s)
                                                                    : launch_pass<double>(c, words, a, s);
            if (rc) return rc;
        }
        if (c->replaying) {
            // the recorded build's counts, checked on the device
            const BuildRecord& r = c->rec;
            AC_TRY(expect_u64(c, &dc->n_pending, (unsigned long long)r.n_pending, s));
            if (r.n_pending > 0) {
                k_resolve_prep<<<resolve_blocks(r.n_pending, 1), 128, 0, s>>>(a, r.n_pending, scan);
                AC_LAUNCHED();
                k_resolve_scan<<<resolve_blocks(r.n_pending, RESOLVE_LANES), 128, 0, s>>>(a, scan);
                AC_LAUNCHED();
            }
            AC_TRY(expect_u64(c, &dc->n_tet_out, r.post.n_tet_out, s));
            AC_TRY(expect_u64(c, &dc->n_tri_pass, r.post.n_tri_pass, s));
            AC_TRY(expect_u64(c, &dc->n_edge_pass, r.post.n_edge_pass, s));
            for (int d = 1; d < 4; d++) AC_TRY(expect_u64(c, &dc->n_cand_out[d], r.post.n_cand_out[d], s));
            c->hc = r.post;
            return AC_OK;
        }
        // the resolve kernels sized by the list's capacity, reading the count on the device: one host wait
        if (c->cap_pending > 0) {
            k_resolve_prep<<<resolve_blocks(c->cap_pending, 1), 128, 0, s>>>(a, -1, scan);
            AC_LAUNCHED();
            k_resolve_scan<<<resolve_blocks(c->cap_pending, RESOLVE_LANES), 128, 0, s>>>(a, scan);
            AC_LAUNCHED();
        }
        AC_TRY(read_counters(c, &h, s));
        if (h.err & DERR_DEGREE) return fail(AC_ERR_CAPACITY, "neighbour list wider than the kernel's masks");
        bool again = false;
        if ((int64_t)h.n_pending > c->cap_pending) {
            c->cap_pending = (int64_t)(h.n_pending * 5 / 4) + 4096;
            again = true;
        }
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
            c->hc = h;
            return AC_OK;
        }
        unsigned zero_err = 0;
        AC_CUDA(cudaMemcpyAsync(&dc->err, &zero_err, sizeof(unsigned), cudaMemcpyHostToDevice, s));
    }
    return fail(AC_ERR_CAPACITY, "output lists kept overflowing");
}

}  // namespace ac
