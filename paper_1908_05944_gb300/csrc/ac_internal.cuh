// Internal declarations of the alphac library (alpha complexes of weighted
// points, arXiv 1908.05944) for sm_103a. Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "alphac.h"

typedef __int128 i128;

namespace ac {

// ---------------------------------------------------------------------------
// error plumbing

void set_detail(const std::string& s);
int fail(int code, const std::string& detail);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define AC_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t _e = (call);                                             \
        if (_e != cudaSuccess) return ac::cuda_fail(_e, #call, __FILE__, __LINE__); \
    } while (0)

// after every kernel launch: check it and count it (reported as kernel_launches)
extern thread_local long long g_launch_count;
#define AC_LAUNCHED()                                                                       \
    do {                                                                                    \
        cudaError_t _e = cudaGetLastError();                                                \
        if (_e != cudaSuccess) return ac::cuda_fail(_e, "kernel launch", __FILE__, __LINE__); \
        ++ac::g_launch_count;                                                               \
    } while (0)

#define AC_TRY(call)            \
    do {                        \
        int _rc = (call);       \
        if (_rc != AC_OK) return _rc; \
    } while (0)

// Device-side error word bits (set with atomicOr by kernels, read by the host).
enum : uint32_t {
    DERR_COINCIDENT = 1u << 0,   // two quantised centres coincide
    DERR_RANGE = 1u << 1,        // a value left the exact-integer range
    DERR_INVALID = 1u << 2,      // NaN/Inf or radius <= 0
    DERR_OVF_TET = 1u << 3,      // K^3 output list full
    DERR_OVF_TRI = 1u << 4,      // unattached-triangle list full
    DERR_OVF_EDGE = 1u << 5,     // unattached-edge list full
    DERR_OVF_CAND = 1u << 6,     // a candidate list full
    DERR_DEGREE = 1u << 7,       // neighbour count above the kernel's mask width
    DERR_INTERNAL = 1u << 8,     // an invariant of the method failed (a bug)
    DERR_OVF_PEND = 1u << 9,     // pending (escalated) list full
    DERR_REPLAY = 1u << 10,      // a size differs from the one recorded for the graph replay
    DERR_TIMEOUT = 1u << 11,     // a bounded device wait ran out
};

// ---------------------------------------------------------------------------
// grow-only device buffer

// Device buffer from the device's stream-ordered memory pool (cudaMallocAsync),
// which keeps freed blocks for reuse by later contexts instead of returning
// them to the driver. Growth and release are ordered on the stream of the
// entry point running (StreamScope), so no device-wide synchronisation is
// needed, and a block is reused only after the work that used it. The buffers
// of a destroyed context (released after a device synchronisation, so idle)
// go to a process-wide cache that later reserves draw on first.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept;
    ~DevBuf();
    int reserve(size_t nbytes, cudaStream_t s);  // keeps contents only if no growth happened
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// The stream on which buffers destroyed on this thread are released; set for
// the duration of an entry point.
cudaStream_t& release_stream();
struct StreamScope {
    cudaStream_t prev;
    explicit StreamScope(cudaStream_t s) : prev(release_stream()) { release_stream() = s; }
    ~StreamScope() { release_stream() = prev; }
};

// ---------------------------------------------------------------------------
// counters written by the kernels (one device struct, zeroed per build)

struct DevCounters {
    unsigned long long n_tet_out;     // K^3 emitted
    unsigned long long n_tri_pass;    // Sigma^2 triangles with AC2 at their orthocentre
    unsigned long long n_edge_pass;   // Sigma^1 edges with AC2
    unsigned long long n_cand[4];     // |Sigma^d| (d = 1..3 counted in the per-atom pass)
    unsigned long long n_cand_out[4]; // candidates written (keep_candidates)
    unsigned long long ac2_tet[3];
    unsigned long long ac2_tri[3];
    unsigned long long ac2_edge;
    unsigned long long ac3[4];
    unsigned long long ac3_exact;     // AC3 decisions left to exact integers
    unsigned long long n_pending;     // simplices escalated to the resolve kernels
    unsigned long long n_scan;        // escalated simplices whose AC3 holds (their AC2 scan list)
    unsigned long long work_next;     // persistent-kernel work counter (narrow-row launch)
    unsigned long long work_next2;    // work counter of the wide-row launch
    unsigned long long work_next3;    // work counter of the launch for atoms beyond 512 neighbours
    unsigned long long work_next4;    // work counters of the launches for 129..256 and 65..128 neighbours
    unsigned long long work_next5;
    unsigned int err;
    int max_degree;
    int bad_index;
    int pad;
    unsigned long long nb_sum;        // neighbour pairs counted (sum of |L(i)|)
};

// Row length of the padded neighbour layout: L(i) at nb[i * NB_STRIDE ..]
// when no atom has more neighbours, else a compact list at scanned offsets.
constexpr int NB_STRIDE = 128;
// Most grown-ball neighbours an atom may have (rows of 32 words of 32 bits,
// 10-bit row positions in the per-atom pass).
constexpr int MAX_DEGREE = 1024;

// Grid of one molecule: origin (quanta), cell side, dims, first global cell.
struct MolGrid {
    int32_t org[3];
    int32_t dims[3];
    int64_t cell_base;
};

// Build-wide constants for the predicates.
struct PredConst {
    int64_t A;        // alpha in quanta^2
    int64_t H2;       // max(W) + A: squared radius bound of a grown ball
    int32_t cell;     // grid cell side in quanta
    int32_t reach;    // cells searched per axis for neighbours: ceil(2h / cell)
    float h_f;        // sqrt(H2) rounded up, FP32
    double h_d;       // sqrt(H2) rounded up, FP64
    int precision;    // AC_PRECISION_*
    int keep_candidates;
};

// One list of simplices of one dimension in canonical order.
struct SimplexList {
    DevBuf tuples;   // int32 (count, d+1), per-molecule local indices
    DevBuf f;        // double
    DevBuf orthosize;// double
    DevBuf attached; // uint8
    DevBuf src_dim;  // int8: dimension of the source simplex (closest witness)
    DevBuf src_idx;  // int64: index of the source simplex in its list
    DevBuf v0_off;   // int64 (n+1): rows with first vertex (global input index) g start at v0_off[g]
    int64_t count = 0;
    std::vector<int64_t> mol_off;  // host: first row of each molecule, n_mol + 1
};

}  // namespace ac

namespace ac {
// Scratch of the canonicalisation, kept by the context so rebuilds allocate nothing.
struct CanonWork {
    DevBuf T, cnt, cursor, uniq, big;
};

// A size a replay checks on the device: *p (kind 0: int64, 1: uint64) equals
// want, or (kind 2) the count int32 at p equal those at ref.
struct ExpectEntry {
    const void* p;
    const void* ref;
    long long want;
    int kind;
    int count;
};
constexpr int MAX_EXPECTS = 64;

// Sizes a synchronised build read back; later builds replay with these.
struct BuildRecord {
    bool valid = false;
    ac_options opt{};
    int wmax = 0;
    int64_t nb_total = 0, n_wide = 0, n_huge = 0, n_w128 = 0, n_w256 = 0;
    int nb_stride = 0;      // layout of the neighbour lists (0: compact)
    int64_t n_pending = 0;  // escalated simplices before the resolve kernel
    DevCounters post{};     // counters after the resolve kernel
    int64_t count[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // K^0..K^3 rows, then Sigma^1..Sigma^3 rows
};
}  // namespace ac

struct ac_ctx {
    int64_t n = 0;
    int64_t n_mol = 1;
    std::vector<int64_t> mol_off;  // host, n_mol + 1
    double alpha = 0.0;
    ac_options opt{};
    ac::PredConst pc{};
    bool built = false;
    bool plan_fresh = false;  // ac_create just quantised and planned; the first build reuses that

    // inputs
    ac::DevBuf centres;  // double n x 3 (input order)
    ac::DevBuf radii;    // double n
    ac::DevBuf P;        // int4 (X, Y, Z, W) quantised, input order
    ac::DevBuf mol_of;   // int32 molecule of each atom (input order)
    ac::DevBuf d_moloff; // int64 n_mol + 1
    ac::DevBuf grids;    // MolGrid per molecule
    std::vector<ac::MolGrid> h_grids;  // host copy (the source of the device copy)
    int64_t n_cells = 0;

    // grid + sorted order
    ac::DevBuf cell_of;   // uint32 per atom (input order)
    ac::DevBuf cell_cnt;  // uint32 per cell
    ac::DevBuf cell_start;// uint32 per cell + 1
    ac::DevBuf order;     // int32: sorted position -> input index
    ac::DevBuf rank;      // int32: input index -> sorted position
    ac::DevBuf Ps;        // int4 sorted
    ac::DevBuf mol_s;     // int32 molecule, sorted

    // neighbour lists (sorted positions)
    // nb_stride == NB_STRIDE: counts in nb_cnt, L(i) at nb[i * NB_STRIDE];
    // nb_stride == 0: nb_cnt holds exclusive offsets (n + 1) into a compact nb
    ac::DevBuf nb_cnt;   // int64 n+1
    ac::DevBuf nb;       // int32
    int64_t nb_total = 0;
    int nb_stride = 0;

    // per-atom pass outputs (sorted positions)
    ac::DevBuf tet_out;   // int4
    ac::DevBuf tri_pass;  // int4 (x,y,z used)
    ac::DevBuf edge_pass; // int2
    ac::DevBuf vert_pass; // uint8 per sorted atom
    ac::DevBuf cand[4];   // Sigma^d candidate lists when kept (int4 / int2)
    ac::DevBuf pending;   // int4 escalated simplices (see ac_local.cu)
    ac::DevBuf resolve_scan;  // their AC2 scan records (ResolveScan, ac_local.cu)
    ac::DevBuf work;      // int32 sorted positions by decreasing neighbour count
    ac::DevBuf deg;       // degree histogram and cursors of the work order
    int64_t n_wide = 0;   // atoms with more than 64 neighbours (the head of work)
    int64_t n_huge = 0;   // atoms with more than 512 neighbours (the head of the head)
    int64_t n_w128 = 0, n_w256 = 0;  // atoms with more than 128, more than 256 neighbours
    ac::DevBuf huge_ws;   // per-warp working sets of the launch for those atoms (global memory)
    int64_t cap_tet = 0, cap_tri = 0, cap_edge = 0, cap_cand[4] = {0, 0, 0, 0}, cap_pending = 0;

    // canonical results; Gbuf/CGbuf hold the same rows as int4 of global input indices
    ac::SimplexList K[4];
    ac::DevBuf Gbuf[4];
    ac::SimplexList C[4];  // Sigma^d (keep_candidates)
    ac::DevBuf CGbuf[4];

    // scratch
    ac::DevBuf counters;  // DevCounters
    ac::DevBuf scratch[7];
    // host copies of the lists (opt.host_results): per dimension one page-locked
    // block [rows int32 | values f64 | attached u8], from a process-wide cache
    void* hres[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t hres_bytes[4] = {0, 0, 0, 0};
    ac::DevBuf fkey[4];      // per-dimension coface-minimum keys (k_orthosize, k_coface_*)
    ac::DevBuf fargs[4];     // per-dimension lexicographic argmin of the coface minimum
    ac::DevBuf frows[4];     // per-dimension facet rows of the cofaces (k_coface_min -> k_coface_arg)
    bool os_forked = false;  // k_orthosize launches on the side stream await their join
    int64_t pair_words = 0;  // words of the triangle pair masks (recorded for replays)
    ac::DevBuf pair_moff;    // first pair-mask word of each sorted position (n + 1)
    ac::DevBuf scan_tmp;

    ac::DevCounters hc{};             // host copy of the counters from the last readback
    void* h_pinned = nullptr;         // one page-locked block holding the four readback areas below
    int64_t* h_stage = nullptr;       // small scalars
    ac::DevCounters* h_cnt = nullptr; // counters
    int32_t* h_bbox = nullptr;        // 6 x n_mol bounding boxes
    int64_t* h_molrows = nullptr;     // 7 x (n_mol + 1) per-molecule first rows

    // graph replay of later builds
    bool replaying = false;       // set while the replay sequence is being captured
    ac::BuildRecord rec;
    ac::DevBuf rec_bbox;          // int32 6 x n_mol: bounding boxes of the recorded build
    cudaStream_t cap_stream = nullptr;  // private stream the replay is captured on (never the legacy stream)
    std::vector<ac::ExpectEntry> expects;  // checks gathered while capturing, run by one kernel at the end
    ac::DevBuf expect_table;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_launches = 0; // kernels in the graph
    int host_syncs = 0;           // host waits in the current build
    ac::CanonWork cw;

    ac_stats stats{};
    int res_device = -1;        // device of the cached CUDA objects below
    size_t h_pinned_bytes = 0;
    cudaEvent_t ev[10] = {};  // stage boundaries; ev[8], ev[9] bracket the per-atom kernel
    cudaStream_t side = nullptr;                    // wide-row launch, concurrent with the narrow one
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t copy = nullptr;                    // host copies of the lists (opt.host_results)
    cudaEvent_t ev_copy = nullptr, ev_cjoin = nullptr;
    bool copy_forked = false;                       // copies on the copy stream await their join
    int local_launches = 0;
};

namespace ac {

// launchers (each returns AC_OK or an AC_ERR_*)
// exclusive scans: n inputs -> n + 1 outputs (out[n] = total); in may alias out
int scan_exclusive_i64(ac_ctx* c, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
int scan_exclusive_u32_to_u32(ac_ctx* c, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);

int quantise_and_plan(ac_ctx* c, cudaStream_t s);
int plan_pair_masks(ac_ctx* c, const int64_t* pw, cudaStream_t s);
// page-locked host block of at least `bytes` for list d's host copy (process-wide cache)
int host_block_for(ac_ctx* c, int d, size_t bytes);
// byte offsets of the three parts of a host block holding `count` rows of k entries
inline size_t hres_f_off(int64_t count, int k) { return ((size_t)count * k * sizeof(int32_t) + 15) & ~(size_t)15; }
inline size_t hres_a_off(int64_t count, int k) { return hres_f_off(count, k) + (size_t)count * sizeof(double); }
inline size_t hres_bytes_for(int64_t count, int k) { return hres_a_off(count, k) + (size_t)count; }

// 32-bit words of an atom's triangle pair mask: one bit per pair of its m neighbours
__device__ __forceinline__ int64_t pair_mask_words(int m) { return ((int64_t)m * (m - 1) / 2 + 31) / 32; }
int build_grid(ac_ctx* c, cudaStream_t s);
int build_neighbours(ac_ctx* c, cudaStream_t s);
int run_local(ac_ctx* c, cudaStream_t s);
int canonicalise(ac_ctx* c, cudaStream_t s);
int compute_filtration(ac_ctx* c, cudaStream_t s);
int eval_filtration(ac_ctx* c, const double* centres, const double* radii, double* const f_out[4], cudaStream_t s);
int eval_filtration_f32(ac_ctx* c, float* const f_out[4], cudaStream_t s);
int backward(ac_ctx* c, const double* const dldf[4], double* dc, double* dr, cudaStream_t s);
int backward_noalloc(ac_ctx* c, const double* const dldf[4], double* dc, double* dr, cudaStream_t s);
int subcomplex_flags(ac_ctx* c, int dim, int64_t first, int64_t m, double alpha2, uint8_t* flags, int64_t* count,
                     cudaStream_t s);

int read_counters(ac_ctx* c, DevCounters* h, cudaStream_t s);
// Replay checks: set DERR_REPLAY in the counters when a device value differs
// from the recorded one.
int expect_i64(ac_ctx* c, const int64_t* d_value, int64_t want, cudaStream_t s);
int expect_u64(ac_ctx* c, const unsigned long long* d_value, unsigned long long want, cudaStream_t s);
int expect_i32s(ac_ctx* c, const int32_t* d_values, const int32_t* d_ref, int64_t count);
int sync_host(ac_ctx* c, cudaStream_t s);  // cudaStreamSynchronize, counted in the build's stats
// Record stage event k; under graph capture as an external event node, so the
// replayed graph records it too.
int stage_mark(ac_ctx* c, int k, cudaStream_t s);
void finish_mol_rows(ac_ctx* c);

// device helpers -------------------------------------------------------------

__host__ __device__ inline int64_t div_floor(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

}  // namespace ac
