// C-ABI entry points of alphac and the host-side orchestration of one build.
// The stages follow the paper (arXiv 1908.05944): grid binning (Section 4.2),
// potential simplices and pruning (Sections 4.3-4.4, Steps 1-5 of Section 3.1),
// then canonical lists and Size filtration values (Section 2.3).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "ac_internal.cuh"

namespace ac {

static thread_local std::string g_detail;
thread_local long long g_launch_count = 0;

void set_detail(const std::string& s) { g_detail = s; }

int fail(int code, const std::string& detail) {
    g_detail = detail;
    return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_detail = buf;
    return e == cudaErrorMemoryAllocation ? AC_ERR_OOM : AC_ERR_CUDA;
}

cudaStream_t& release_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}

// Set while a replay is captured: every buffer must already have its size.
static thread_local bool g_no_alloc = false;

// Keep up to this many freed bytes per device in the pool between builds.
static constexpr uint64_t POOL_KEEP_BYTES = 16ull << 30;

static void prepare_pool() {
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> g(mu);
    for (int d : done)
        if (d == dev) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = POOL_KEEP_BYTES;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done.push_back(dev);
}

// Device blocks of destroyed contexts. ac_destroy synchronises the device
// before it releases a context's buffers, so a block released then is idle and
// may serve a later reserve on any stream: the next context of a similar size
// takes its buffers from here instead of from the stream-ordered allocator
// (an allocation call per buffer).
struct IdleBlock {
    void* p;
    int dev;
};
static std::mutex g_idle_mu;
static std::multimap<size_t, IdleBlock> g_idle;  // by size
static size_t g_idle_bytes = 0;
// Only blocks up to IDLE_MAX_BLOCK are kept: the allocation calls saved are per
// buffer, and a large block held here is memory the pool cannot hand to a
// context of another size.
static constexpr size_t IDLE_KEEP_BYTES = 2ull << 30;
static constexpr size_t IDLE_MAX_BLOCK = 64ull << 20;
static constexpr size_t IDLE_KEEP_BLOCKS = 1024;
static thread_local bool g_release_idle = false;  // set by ac_destroy once the device is idle

static bool idle_give(void* p, size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (bytes > IDLE_MAX_BLOCK) return false;
    std::lock_guard<std::mutex> g(g_idle_mu);
    if (g_idle_bytes + bytes > IDLE_KEEP_BYTES || g_idle.size() >= IDLE_KEEP_BLOCKS) return false;
    g_idle.emplace(bytes, IdleBlock{p, dev});
    g_idle_bytes += bytes;
    return true;
}

// The smallest idle block of this device with want..2 want + 1 MB bytes, or null.
static void* idle_take(size_t want, size_t* got) {
    if (want > IDLE_MAX_BLOCK) return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(g_idle_mu);
    const size_t limit = 2 * want + (1u << 20);
    for (auto it = g_idle.lower_bound(want); it != g_idle.end() && it->first <= limit; ++it) {
        if (it->second.dev != dev) continue;
        void* p = it->second.p;
        *got = it->first;
        g_idle_bytes -= it->first;
        g_idle.erase(it);
        return p;
    }
    return nullptr;
}

DevBuf::~DevBuf() {
    if (p && !(g_release_idle && idle_give(p, bytes))) cudaFreeAsync(p, release_stream());
}

DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
    if (this != &o) {
        if (p) cudaFreeAsync(p, release_stream());
        p = o.p;
        bytes = o.bytes;
        o.p = nullptr;
        o.bytes = 0;
    }
    return *this;
}

int DevBuf::reserve(size_t nbytes, cudaStream_t s) {
    if (nbytes <= bytes && p) return AC_OK;
    if (g_no_alloc) return fail(AC_ERR_STATE, "a buffer would grow during graph capture");
    if (p) {
        cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    size_t want = nbytes < 256 ? 256 : nbytes;
    size_t got = 0;
    if (void* q = idle_take(want, &got)) {
        p = q;
        bytes = got;
        return AC_OK;
    }
    prepare_pool();
    cudaError_t e = cudaMallocAsync(&p, want, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        char buf[128];
        snprintf(buf, sizeof(buf), "cudaMallocAsync of %zu bytes failed", want);
        return fail(AC_ERR_OOM, buf);
    }
    bytes = want;
    return AC_OK;
}

// ---------------------------------------------------------------------------
// exclusive scan (n inputs -> n + 1 outputs, out[n] = total); in may alias out

template <class T>
__device__ inline T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ T block_excl_scan(T v, T* total) {
    __shared__ T warp_sums[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_sums[lane] : T(0);
        T wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    T r = inc - v + warp_sums[wid];
    __syncthreads();
    return r;
}

// Single-pass exclusive scan (decoupled look-back): tiles take their index
// from a counter in launch order, publish their sum, then add the sums (or the
// inclusive prefix, once known) of the tiles before them. A tile only waits
// on tiles that took an earlier index and are therefore running; the wait is
// bounded all the same. When it runs out (spin_limit polls of one tile's
// flag), the tile sets DERR_TIMEOUT and sums that predecessor's inputs itself,
// so the offsets stay exact and no later kernel writes where it should not:
// a predecessor that has not published its sum has not written its outputs
// either (it writes them after publishing), which is checked again after the
// sum, so this holds for in-place scans too. The build still reports
// AC_ERR_TIMEOUT, and the context stays usable.
constexpr long long SCAN_SPIN_LIMIT = 1ll << 24;  // polls per flag: far beyond any real wait (microseconds)

struct ScanState {
    unsigned next_tile;
    unsigned pad;
};

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_lookback(const T* in, T* out, int64_t n, ScanState* st,
                                                                 int* flags, T* agg, T* inc, unsigned* err,
                                                                 long long spin_limit) {
    __shared__ int tile_s;
    __shared__ T prefix_s;
    __shared__ T total_s;
    if (threadIdx.x == 0) tile_s = (int)atomicAdd(&st->next_tile, 1u);
    __syncthreads();
    const int tile = tile_s;
    const int64_t base = (int64_t)tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const int64_t i = base + k;
        v[k] = i < n ? in[i] : T(0);
        sum += v[k];
    }
    T pre = block_excl_scan<T>(sum, &total_s);  // prefix within the tile
    if (threadIdx.x == 0) {
        const T total = total_s;
        volatile int* vf = flags;
        T acc = 0;
        if (tile == 0) {
            inc[0] = total;
            __threadfence();
            vf[0] = 2;
        } else {
            agg[tile] = total;
            __threadfence();
            vf[tile] = 1;
            int p = tile - 1;
            long long spins = 0;
            bool force = spin_limit < 0;  // a negative limit: take the path below once, whatever the flag
            while (p >= 0) {
                int f = vf[p];
                if (f == 0 || force) {
                    if (!force && spins++ < spin_limit) continue;
                    force = false;
                    // the wait ran out: sum tile p's inputs here, then keep
                    // that sum unless p has published in the meantime
                    atomicOr(err, DERR_TIMEOUT);
                    T own = 0;
                    const int64_t b0 = (int64_t)p * SCAN_TILE;
                    for (int64_t i = b0; i < b0 + SCAN_TILE && i < n; i++) own += __ldcg(in + i);
                    __threadfence();
                    f = vf[p];
                    spins = 0;
                    if (f == 0) {
                        acc += own;
                        p--;
                        continue;
                    }
                }
                __threadfence();
                if (f == 2) {
                    acc += *(volatile T*)&inc[p];
                    break;
                }
                acc += *(volatile T*)&agg[p];
                spins = 0;
                p--;
            }
            inc[tile] = acc + total;
            __threadfence();
            vf[tile] = 2;
        }
        prefix_s = acc;
    }
    __syncthreads();
    pre += prefix_s;
    // out has n + 1 entries: out[n] is the total (the inputs past n count as 0)
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const int64_t i = base + k;
        if (i <= n) out[i] = pre;
        pre += v[k];
    }
}

// Two-pass scan for up to SCAN_SMALL_TILES tiles (4 M elements): the tile
// sums, then every tile adds up the sums before it (at most a few thousand
// values) and scans itself. No tile waits on another.
constexpr int64_t SCAN_SMALL_TILES = 1024;

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(const T* in, int64_t n, T* agg) {
    __shared__ T total_s;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const int64_t i = base + k;
        if (i < n) sum += in[i];
    }
    block_excl_scan<T>(sum, &total_s);
    if (threadIdx.x == 0) agg[blockIdx.x] = total_s;
}

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const T* in, T* out, int64_t n, const T* agg) {
    __shared__ T before_s;
    __shared__ T total_s;
    T p = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += SCAN_THREADS) p += agg[t];
    block_excl_scan<T>(p, &before_s);  // before_s: the sum of the tiles before this one
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const int64_t i = base + k;
        v[k] = i < n ? in[i] : T(0);
        sum += v[k];
    }
    T pre = block_excl_scan<T>(sum, &total_s) + before_s;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        const int64_t i = base + k;
        if (i <= n) out[i] = pre;
        pre += v[k];
    }
}

// Polls of one flag before a look-back tile stops waiting: SCAN_SPIN_LIMIT, or
// the value of the environment variable ALPHAC_SCAN_SPIN_LIMIT (read at every
// launch): 0 stops at the first unpublished flag, and a negative value makes
// every tile take that path once, for its nearest predecessor (a test of it).
static long long scan_spin_limit() {
    const char* e = getenv("ALPHAC_SCAN_SPIN_LIMIT");
    if (!e || !*e) return SCAN_SPIN_LIMIT;
    char* end = nullptr;
    const long long v = strtoll(e, &end, 10);
    return (end && *end == '\0') ? v : SCAN_SPIN_LIMIT;
}

template <class T>
static int scan_entry(const T* in, T* out, int64_t n, DevBuf& tmp, DevCounters* dc, cudaStream_t s) {
    if (n <= 0) {
        AC_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
        return AC_OK;
    }
    const int64_t tiles = n / SCAN_TILE + 1;  // n + 1 outputs
    if (tiles <= SCAN_SMALL_TILES) {
        AC_TRY(tmp.reserve((size_t)tiles * sizeof(T), s));
        k_scan_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, tmp.as<T>());
        AC_LAUNCHED();
        k_scan_tiles<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, tmp.as<T>());
        AC_LAUNCHED();
        return AC_OK;
    }
    // state: counter, flags (int per tile), aggregates and inclusive prefixes (T per tile)
    const size_t flags_off = 64, agg_off = (flags_off + (size_t)tiles * sizeof(int) + 63) & ~(size_t)63;
    const size_t inc_off = (agg_off + (size_t)tiles * sizeof(T) + 63) & ~(size_t)63;
    const size_t need = inc_off + (size_t)tiles * sizeof(T);
    AC_TRY(tmp.reserve(need, s));
    char* b = static_cast<char*>(tmp.p);
    AC_CUDA(cudaMemsetAsync(b, 0, agg_off, s));  // counter and flags
    k_scan_lookback<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, reinterpret_cast<ScanState*>(b),
                                                                 reinterpret_cast<int*>(b + flags_off),
                                                                 reinterpret_cast<T*>(b + agg_off),
                                                                 reinterpret_cast<T*>(b + inc_off), &dc->err,
                                                                 scan_spin_limit());
    AC_LAUNCHED();
    return AC_OK;
}

int scan_exclusive_i64(ac_ctx* c, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_entry<long long>(reinterpret_cast<const long long*>(in), reinterpret_cast<long long*>(out), n,
                                 c->scan_tmp, c->counters.as<DevCounters>(), s);
}

int scan_exclusive_u32_to_u32(ac_ctx* c, const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
    return scan_entry<unsigned>(in, out, n, c->scan_tmp, c->counters.as<DevCounters>(), s);
}

int sync_host(ac_ctx* c, cudaStream_t s) {
    c->host_syncs++;
    AC_CUDA(cudaStreamSynchronize(s));
    return AC_OK;
}

// One thread per check gathered during the capture (they all read values
// that stay in place until the end of the build).
__global__ void k_check_expects(const ExpectEntry* __restrict__ t, int n, unsigned* __restrict__ err) {
    const int j = threadIdx.x;
    if (j >= n) return;
    const ExpectEntry e = t[j];
    bool ok = true;
    if (e.kind == 0) ok = *static_cast<const long long*>(e.p) == e.want;
    else if (e.kind == 1) ok = *static_cast<const unsigned long long*>(e.p) == (unsigned long long)e.want;
    else {
        const int32_t* a = static_cast<const int32_t*>(e.p);
        const int32_t* b = static_cast<const int32_t*>(e.ref);
        for (int k = 0; k < e.count && ok; k++) ok = a[k] == b[k];
    }
    if (!ok) atomicOr(err, DERR_REPLAY);
}

int stage_mark(ac_ctx* c, int k, cudaStream_t s) {
    AC_CUDA(cudaEventRecordWithFlags(c->ev[k], s, c->replaying ? cudaEventRecordExternal : cudaEventRecordDefault));
    return AC_OK;
}

static int add_expect(ac_ctx* c, const ExpectEntry& e) {
    if ((int)c->expects.size() >= MAX_EXPECTS) return fail(AC_ERR_CAPACITY, "too many replay checks");
    c->expects.push_back(e);
    return AC_OK;
}

int expect_i64(ac_ctx* c, const int64_t* d_value, int64_t want, cudaStream_t) {
    return add_expect(c, ExpectEntry{d_value, nullptr, (long long)want, 0, 1});
}

int expect_u64(ac_ctx* c, const unsigned long long* d_value, unsigned long long want, cudaStream_t) {
    return add_expect(c, ExpectEntry{d_value, nullptr, (long long)want, 1, 1});
}

int expect_i32s(ac_ctx* c, const int32_t* d_values, const int32_t* d_ref, int64_t count) {
    if (count > INT32_MAX) return fail(AC_ERR_CAPACITY, "replay check too long");
    return add_expect(c, ExpectEntry{d_values, d_ref, 0, 2, (int)count});
}

int read_counters(ac_ctx* c, DevCounters* h, cudaStream_t s) {
    AC_CUDA(cudaMemcpyAsync(c->h_cnt, c->counters.p, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    AC_TRY(sync_host(c, s));
    *h = *c->h_cnt;
    c->hc = *h;
    return AC_OK;
}

// ---------------------------------------------------------------------------
// quantisation (input order) and per-molecule bounding boxes

__global__ void k_quantise(const double* __restrict__ centres, const double* __restrict__ radii, int64_t n,
                           const int32_t* __restrict__ mol_of, int4* __restrict__ P, int32_t* __restrict__ bbox,
                           int* __restrict__ wmax, DevCounters* cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    bool ok = false;
    int X = 0, Y = 0, Z = 0, W = 0, m = -1;
    if (i < n) {
        double x = centres[3 * i], y = centres[3 * i + 1], z = centres[3 * i + 2], r = radii[i];
        bool finite = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(r);
        const double lim = 1048576.0;  // |x| <= 2^20 A: the quantised coordinate fits 32 bits
        uint32_t bad = 0;
        if (!finite || !(r > 0.0)) {
            bad = DERR_INVALID;
        } else if (fabs(x) > lim || fabs(y) > lim || fabs(z) > lim || r > 64.0) {
            bad = DERR_RANGE;
        } else {
            X = __double2int_rn(x * 1024.0);
            Y = __double2int_rn(y * 1024.0);
            Z = __double2int_rn(z * 1024.0);
            const int R = __double2int_rn(r * 1024.0);
            // |X| < 2^30 keeps every difference of two coordinates (a grid offset) within 32 bits;
            // a radius quantised to 0, or above 4 A, would take W out of the 2^24 range of the predicates
            const int cmax = (1 << 30) - 1;
            if (X > cmax || X < -cmax || Y > cmax || Y < -cmax || Z > cmax || Z < -cmax || R < 1 || R > 4096)
                bad = DERR_RANGE;
            else W = R * R;
        }
        if (bad) {
            atomicOr(&cnt->err, bad);
            atomicMin(&cnt->bad_index, (int)i);
        } else {
            P[i] = make_int4(X, Y, Z, W);
            ok = true;
            m = mol_of[i];
        }
    }
    // bounds reduced per warp when its atoms share a molecule (the usual case), then per block
    // when all of its warps do: one set of atomics per block instead of one per atom
    __shared__ int red[8][8];  // per warp: molecule (-1: none, -2: mixed), min x y z, max x y z, max W
    const int wid = threadIdx.x >> 5;
    const int m0 = __shfl_sync(full, m, 0);
    const bool uniform = __all_sync(full, !ok || m == m0) && __any_sync(full, ok);
    const int big = 0x7fffffff, small = (int)0x80000000;
    int v[8];
    if (uniform) {
        v[0] = __reduce_max_sync(full, m);
        v[1] = __reduce_min_sync(full, ok ? X : big);
        v[2] = __reduce_min_sync(full, ok ? Y : big);
        v[3] = __reduce_min_sync(full, ok ? Z : big);
        v[4] = __reduce_max_sync(full, ok ? X : small);
        v[5] = __reduce_max_sync(full, ok ? Y : small);
        v[6] = __reduce_max_sync(full, ok ? Z : small);
        v[7] = __reduce_max_sync(full, ok ? W : 0);
    } else {
        v[0] = __any_sync(full, ok) ? -2 : -1;
    }
    if (lane == 0)
        for (int k = 0; k < 8; k++) red[wid][k] = v[k];
    __syncthreads();
    const int nw = blockDim.x >> 5;  // 256-thread blocks: 8 warps
    int bm = -1;                      // the block's molecule, or -2 if its warps differ
    for (int w = 0; w < nw; w++) {
        const int mw = red[w][0];
        if (mw == -1) continue;
        bm = (bm == -1 && mw >= 0) ? mw : (bm == mw ? bm : -2);
    }
    if (bm >= 0) {
        if (threadIdx.x == 0) {
            int r[8] = {bm, big, big, big, small, small, small, 0};
            for (int w = 0; w < nw; w++) {
                if (red[w][0] < 0) continue;
                for (int k = 1; k <= 3; k++) r[k] = min(r[k], red[w][k]);
                for (int k = 4; k <= 7; k++) r[k] = max(r[k], red[w][k]);
            }
            int32_t* b = bbox + 6 * bm;
            atomicMin(&b[0], r[1]);
            atomicMin(&b[1], r[2]);
            atomicMin(&b[2], r[3]);
            atomicMax(&b[3], r[4]);
            atomicMax(&b[4], r[5]);
            atomicMax(&b[5], r[6]);
            atomicMax(wmax, r[7]);
        }
    } else if (uniform) {
        if (lane == 0) {
            int32_t* b = bbox + 6 * v[0];
            atomicMin(&b[0], v[1]);
            atomicMin(&b[1], v[2]);
            atomicMin(&b[2], v[3]);
            atomicMax(&b[3], v[4]);
            atomicMax(&b[4], v[5]);
            atomicMax(&b[5], v[6]);
            atomicMax(wmax, v[7]);
        }
    } else if (ok) {
        int32_t* b = bbox + 6 * m;
        atomicMin(&b[0], X);
        atomicMin(&b[1], Y);
        atomicMin(&b[2], Z);
        atomicMax(&b[3], X);
        atomicMax(&b[4], Y);
        atomicMax(&b[5], Z);
        atomicMax(wmax, W);
    }
}

__global__ void k_fill_mol(const int64_t* __restrict__ mol_off, int64_t n_mol, int32_t* __restrict__ mol_of) {
    int64_t m = blockIdx.x;
    if (m >= n_mol) return;
    for (int64_t i = mol_off[m] + threadIdx.x; i < mol_off[m + 1]; i += blockDim.x) mol_of[i] = (int32_t)m;
}

__global__ void k_init_bbox(int32_t* bbox, int64_t n_mol, DevCounters* cnt) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m == 0) cnt->bad_index = INT32_MAX;
    if (m >= n_mol) return;
    for (int k = 0; k < 3; k++) {
        bbox[6 * m + k] = INT32_MAX;
        bbox[6 * m + 3 + k] = INT32_MIN;
    }
}

// Quantise the stored inputs (row a1: X = round(1024 x), W = round(1024 r)^2),
// check their ranges, and lay out the per-molecule grids (Section 4.2): cell
// side ~ h = sqrt(r_max^2 + alpha), dense cell table over each bounding box.
int quantise_and_plan(ac_ctx* c, cudaStream_t s) {
    const int64_t n = c->n, n_mol = c->n_mol;
    AC_TRY(c->scratch[0].reserve((size_t)n_mol * 6 * sizeof(int32_t), s));
    AC_TRY(c->scratch[1].reserve(sizeof(int), s));
    DevCounters* dc = c->counters.as<DevCounters>();
    AC_CUDA(cudaMemsetAsync(dc, 0, sizeof(DevCounters), s));
    int32_t* bbox = c->scratch[0].as<int32_t>();
    int* wmax = c->scratch[1].as<int>();
    AC_CUDA(cudaMemsetAsync(wmax, 0, sizeof(int), s));
    k_init_bbox<<<(unsigned)((n_mol + 255) / 256), 256, 0, s>>>(bbox, n_mol, dc);
    AC_LAUNCHED();
    if (n > 0) {
        k_quantise<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c->centres.as<double>(), c->radii.as<double>(), n,
                                                              c->mol_of.as<int32_t>(), c->P.as<int4>(), bbox, wmax, dc);
        AC_LAUNCHED();
    }
    if (c->replaying) {
        // the recorded plan stands; check the bounds it rests on
        AC_TRY(expect_i32s(c, bbox, c->rec_bbox.as<int32_t>(), n_mol * 6));
        AC_TRY(expect_i32s(c, wmax, c->rec_bbox.as<int32_t>() + n_mol * 6, 1));
        return AC_OK;
    }
    // one readback: counters, largest weight, per-molecule boxes
    AC_CUDA(cudaMemcpyAsync(c->h_cnt, c->counters.p, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    AC_CUDA(cudaMemcpyAsync(c->h_stage, wmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    AC_CUDA(cudaMemcpyAsync(c->h_bbox, bbox, (size_t)n_mol * 6 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    AC_TRY(sync_host(c, s));
    const DevCounters hc = *c->h_cnt;
    if (hc.err & DERR_INVALID) {
        char b[128];
        snprintf(b, sizeof(b), "atom %d: non-finite value or radius <= 0", hc.bad_index);
        return fail(AC_ERR_INVALID_ARG, b);
    }
    if (hc.err & DERR_RANGE) {
        char b[160];
        snprintf(b, sizeof(b), "atom %d: |coordinate| >= 2^20 A or radius outside (0, 4] A after quantisation",
                 hc.bad_index);
        return fail(AC_ERR_RANGE, b);
    }
    const int wmax_h = *reinterpret_cast<const int*>(c->h_stage);
    const int32_t* hb = c->h_bbox;

    PredConst& pc = c->pc;
    pc.A = (int64_t)nearbyint(c->alpha * 1048576.0);
    pc.H2 = (int64_t)wmax_h + pc.A;
    if (pc.H2 > ((int64_t)1 << 24)) return fail(AC_ERR_RANGE, "r_max^2 + alpha exceeds 16 A^2");
    pc.precision = c->opt.precision;
    pc.keep_candidates = c->opt.keep_candidates ? 1 : 0;
    int64_t hq = 0;  // ceil(sqrt(H2)) in quanta
    if (pc.H2 > 0) {
        hq = (int64_t)floor(sqrt((double)pc.H2));
        while (hq * hq < pc.H2) hq++;
    }
    pc.h_f = (float)hq;
    pc.h_d = (double)hq;
    int64_t cell = (int64_t)ceil(c->opt.cell_factor * (double)(hq > 0 ? hq : 1024));
    if (cell < 1) cell = 1;
    // grid dims; coarsen if the dense table would be far larger than the atom count
    std::vector<MolGrid>& grids = c->h_grids;
    grids.assign((size_t)n_mol, MolGrid{});
    int64_t total = 0;
    for (int iter = 0; iter < 40; iter++) {
        total = 0;
        for (int64_t m = 0; m < n_mol; m++) {
            MolGrid& g = grids[(size_t)m];
            bool empty = c->mol_off[(size_t)m + 1] == c->mol_off[(size_t)m];
            for (int k = 0; k < 3; k++) {
                g.org[k] = empty ? 0 : hb[(size_t)(6 * m + k)];
                int64_t span = empty ? 0 : (int64_t)hb[(size_t)(6 * m + 3 + k)] - hb[(size_t)(6 * m + k)];
                g.dims[k] = (int32_t)(span / cell + 1);
            }
            g.cell_base = total;
            total += (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
        }
        if (total <= 16 * n + (1 << 22)) break;
        cell *= 2;
    }
    pc.cell = (int32_t)cell;
    pc.reach = hq > 0 ? (int32_t)((2 * hq + cell - 1) / cell) : 1;
    if (pc.reach < 1) pc.reach = 1;
    c->n_cells = total;
    AC_TRY(c->grids.reserve((size_t)n_mol * sizeof(MolGrid), s));
    // from pageable memory: the call returns once the source is staged, so the
    // next plan may overwrite the host copy
    AC_CUDA(cudaMemcpyAsync(c->grids.p, grids.data(), (size_t)n_mol * sizeof(MolGrid), cudaMemcpyHostToDevice, s));
    c->stats.grid_dims[0] = grids[0].dims[0];
    c->stats.grid_dims[1] = grids[0].dims[1];
    c->stats.grid_dims[2] = grids[0].dims[2];
    c->stats.n_atoms = n;
    return AC_OK;
}

}  // namespace ac

using namespace ac;

// ---------------------------------------------------------------------------
// public API

// The CUDA objects of a context (timing events, fork/join events, the side and
// capture streams, the page-locked readback block) come from a small
// process-wide cache: creating and destroying them costs more than a small
// build, and applications create contexts one after another. A destroyed
// context's objects are idle (ac_destroy synchronises the device first).
struct CtxRes {
    int device = -1;
    cudaEvent_t ev[10] = {};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_copy = nullptr, ev_cjoin = nullptr;
    cudaStream_t side = nullptr, cap_stream = nullptr, copy = nullptr;
    void* pinned = nullptr;
    size_t pinned_bytes = 0;
};

static std::mutex g_res_mu;
static std::vector<CtxRes> g_res;  // at most RES_CACHE entries
constexpr size_t RES_CACHE = 8;

static void res_free(CtxRes& r) {
    for (int k = 0; k < 10; k++)
        if (r.ev[k]) cudaEventDestroy(r.ev[k]);
    if (r.ev_fork) cudaEventDestroy(r.ev_fork);
    if (r.ev_join) cudaEventDestroy(r.ev_join);
    if (r.ev_copy) cudaEventDestroy(r.ev_copy);
    if (r.ev_cjoin) cudaEventDestroy(r.ev_cjoin);
    if (r.side) cudaStreamDestroy(r.side);
    if (r.copy) cudaStreamDestroy(r.copy);
    if (r.cap_stream) cudaStreamDestroy(r.cap_stream);
    if (r.pinned) cudaFreeHost(r.pinned);
    r = CtxRes{};
}

// a cached set for this device with at least pinned_bytes of readback block, or a new one
static int res_take(size_t pinned_bytes, CtxRes& out) {
    int dev = 0;
    AC_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        for (size_t k = 0; k < g_res.size(); k++)
            if (g_res[k].device == dev && g_res[k].pinned_bytes >= pinned_bytes) {
                out = g_res[k];
                g_res.erase(g_res.begin() + (long)k);
                return AC_OK;
            }
    }
    CtxRes r;
    r.device = dev;
    bool ok = true;
    for (int k = 0; k < 10 && ok; k++) ok = cudaEventCreate(&r.ev[k]) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&r.ev_fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&r.ev_join, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&r.ev_copy, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&r.ev_cjoin, cudaEventDisableTiming) == cudaSuccess &&
         cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&r.copy, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&r.cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaMallocHost(&r.pinned, pinned_bytes) == cudaSuccess;
    if (!ok) {
        const cudaError_t e = cudaGetLastError();
        res_free(r);
        return cuda_fail(e, "context events, streams or page-locked block", __FILE__, __LINE__);
    }
    r.pinned_bytes = pinned_bytes;
    out = r;
    return AC_OK;
}

static void res_give(CtxRes& r) {
    if (r.device < 0) return;
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        if (g_res.size() < RES_CACHE) {
            g_res.push_back(r);
            r = CtxRes{};
            return;
        }
    }
    res_free(r);
}

// Page-locked host blocks for the host copies of the lists: pinning memory costs
// far more than a build, so blocks return to a process-wide cache (up to 8 GB)
// when a context is destroyed or needs a larger one, and are taken best-fit.
static std::mutex g_hb_mu;
static std::vector<std::pair<void*, size_t>> g_hb;
static size_t g_hb_total = 0;
constexpr size_t HB_CACHE_BYTES = (size_t)8 << 30;

static void host_block_give(void* p, size_t bytes) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_hb_mu);
        if (g_hb_total + bytes <= HB_CACHE_BYTES) {
            g_hb.emplace_back(p, bytes);
            g_hb_total += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

int ac::host_block_for(ac_ctx* c, int d, size_t bytes) {
    if (c->hres_bytes[d] >= bytes && c->hres[d]) return AC_OK;
    host_block_give(c->hres[d], c->hres_bytes[d]);
    c->hres[d] = nullptr;
    c->hres_bytes[d] = 0;
    {
        std::lock_guard<std::mutex> lk(g_hb_mu);
        size_t best = g_hb.size();
        for (size_t k = 0; k < g_hb.size(); k++)
            if (g_hb[k].second >= bytes && g_hb[k].second <= 4 * bytes + (1 << 20) &&
                (best == g_hb.size() || g_hb[k].second < g_hb[best].second))
                best = k;
        if (best < g_hb.size()) {
            c->hres[d] = g_hb[best].first;
            c->hres_bytes[d] = g_hb[best].second;
            g_hb_total -= g_hb[best].second;
            g_hb.erase(g_hb.begin() + (long)best);
            return AC_OK;
        }
    }
    // a new block, with room to grow (a quarter more, at least 1 MB)
    const size_t want = std::max(bytes + bytes / 4, (size_t)1 << 20);
    if (cudaMallocHost(&c->hres[d], want) != cudaSuccess) {
        c->hres[d] = nullptr;
        return cuda_fail(cudaGetLastError(), "cudaMallocHost of a host result block", __FILE__, __LINE__);
    }
    c->hres_bytes[d] = want;
    return AC_OK;
}

static int create_impl(const double* centres, const double* radii, const int64_t* offsets, int64_t n_mol,
                       double alpha, const ac_options* opt, ac_ctx** out) {
    if (!out) return fail(AC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_mol < 1 || !offsets) return fail(AC_ERR_INVALID_ARG, "need at least one molecule");
    if (offsets[0] != 0) return fail(AC_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int64_t m = 0; m < n_mol; m++)
        if (offsets[m + 1] < offsets[m]) return fail(AC_ERR_INVALID_ARG, "offsets must be non-decreasing");
    int64_t n = offsets[n_mol];
    if (n < 0 || n >= ((int64_t)1 << 31) - 1) return fail(AC_ERR_INVALID_ARG, "n out of range");
    if (n > 0 && (!centres || !radii)) return fail(AC_ERR_INVALID_ARG, "centres/radii NULL");
    if (!isfinite(alpha)) return fail(AC_ERR_INVALID_ARG, "alpha not finite");
    if (fabs(alpha) > 16.0) return fail(AC_ERR_RANGE, "|alpha| must be at most 16 A^2");

    ac_ctx* c = new (std::nothrow) ac_ctx();
    if (!c) return fail(AC_ERR_OOM, "host allocation failed");
    c->n = n;
    c->n_mol = n_mol;
    c->mol_off.assign(offsets, offsets + n_mol + 1);
    c->alpha = alpha;
    if (opt) c->opt = *opt;
    if (c->opt.cell_factor <= 0.0) c->opt.cell_factor = 1.0;
    if (c->opt.block_warps <= 0) c->opt.block_warps = 8;
    if (c->opt.precision != AC_PRECISION_FILTERED && c->opt.precision != AC_PRECISION_PLAIN_FP64) {
        delete c;
        return fail(AC_ERR_INVALID_ARG, "unknown precision mode");
    }
    int rc = AC_OK;
    cudaStream_t s = 0;
    auto bail = [&](int code) {
        ac_destroy(c);
        return code;
    };
    {
        const size_t a0 = 64 * sizeof(int64_t), a1 = (sizeof(DevCounters) + 255) & ~(size_t)255;
        const size_t a2 = ((size_t)6 * n_mol * sizeof(int32_t) + 255) & ~(size_t)255;
        const size_t a3 = (size_t)7 * (n_mol + 1) * sizeof(int64_t);
        // small blocks share one size class, so cached sets fit most contexts
        const size_t need = std::max<size_t>(a0 + a1 + a2 + a3, 64 * 1024);
        CtxRes r;
        if ((rc = res_take(need, r))) return bail(rc);
        for (int k = 0; k < 10; k++) c->ev[k] = r.ev[k];
        c->ev_fork = r.ev_fork;
        c->ev_join = r.ev_join;
        c->ev_copy = r.ev_copy;
        c->ev_cjoin = r.ev_cjoin;
        c->side = r.side;
        c->copy = r.copy;
        c->cap_stream = r.cap_stream;
        c->h_pinned = r.pinned;
        c->h_pinned_bytes = r.pinned_bytes;
        c->res_device = r.device;
        char* b = static_cast<char*>(c->h_pinned);
        c->h_stage = reinterpret_cast<int64_t*>(b);
        c->h_cnt = reinterpret_cast<DevCounters*>(b + a0);
        c->h_bbox = reinterpret_cast<int32_t*>(b + a0 + a1);
        c->h_molrows = reinterpret_cast<int64_t*>(b + a0 + a1 + a2);
    }

    size_t nn = (size_t)(n > 0 ? n : 1);
    if ((rc = c->centres.reserve(nn * 3 * sizeof(double), s)) || (rc = c->radii.reserve(nn * sizeof(double), s)) ||
        (rc = c->P.reserve(nn * sizeof(int4), s)) || (rc = c->mol_of.reserve(nn * sizeof(int32_t), s)) ||
        (rc = c->d_moloff.reserve((size_t)(n_mol + 1) * sizeof(int64_t), s)) ||
        (rc = c->counters.reserve(sizeof(DevCounters), s)))
        return bail(rc);
    // stream-ordered copies: the quantisation below waits for its bounds before ac_create
    // returns, so the caller's buffers are free again by then
    if (n > 0) {
        if (cudaMemcpyAsync(c->centres.p, centres, (size_t)n * 3 * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess ||
            cudaMemcpyAsync(c->radii.p, radii, (size_t)n * sizeof(double), cudaMemcpyDefault, s) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "copy of centres/radii", __FILE__, __LINE__));
    }
    if (cudaMemcpyAsync(c->d_moloff.p, offsets, (size_t)(n_mol + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "copy of offsets", __FILE__, __LINE__));

    k_fill_mol<<<(unsigned)n_mol, 256, 0, s>>>(c->d_moloff.as<int64_t>(), n_mol, c->mol_of.as<int32_t>());
    if (cudaGetLastError() != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "k_fill_mol", __FILE__, __LINE__));
    if ((rc = quantise_and_plan(c, s))) return bail(rc);
    c->plan_fresh = true;
    *out = c;
    return AC_OK;
}

extern "C" int ac_create(const double* centres, const double* radii, int64_t n, double alpha, const ac_options* opt,
                         ac_ctx** out) {
    if (!out) return fail(AC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0) return fail(AC_ERR_INVALID_ARG, "n < 0");
    int64_t off[2] = {0, n};
    return create_impl(centres, radii, off, 1, alpha, opt, out);
}

extern "C" int ac_create_batch(const double* centres, const double* radii, const int64_t* offsets, int64_t n_mol,
                               double alpha, const ac_options* opt, ac_ctx** out) {
    return create_impl(centres, radii, offsets, n_mol, alpha, opt, out);
}

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();  // a stage time is a statistic: leave no error behind
        return -1.f;
    }
    return ms;
}

// The whole path on one stream: rows a1-a13 in order.
static int build_body(ac_ctx* c, cudaStream_t s) {
    AC_TRY(stage_mark(c, 0, s));
    // the inputs were quantised and the grid planned by ac_create: a first
    // build does not repeat it (every later build, replayed or not, does)
    if (c->plan_fresh && !c->replaying) c->plan_fresh = false;
    else AC_TRY(quantise_and_plan(c, s));
    AC_TRY(build_grid(c, s));
    AC_TRY(stage_mark(c, 1, s));
    AC_TRY(build_neighbours(c, s));
    AC_TRY(stage_mark(c, 2, s));
    AC_TRY(run_local(c, s));
    AC_TRY(stage_mark(c, 3, s));
    AC_TRY(canonicalise(c, s));
    AC_TRY(stage_mark(c, 6, s));
    AC_TRY(compute_filtration(c, s));
    if (c->replaying && !c->expects.empty()) {
        // every recorded size, checked once the build's values are in place
        k_check_expects<<<1, MAX_EXPECTS, 0, s>>>(c->expect_table.as<ExpectEntry>(), (int)c->expects.size(),
                                                  &c->counters.as<DevCounters>()->err);
        AC_LAUNCHED();
    }
    AC_TRY(stage_mark(c, 7, s));
    return AC_OK;
}

static bool same_plan(const ac_options& a, const ac_options& b) {
    return a.precision == b.precision && a.filtration == b.filtration && a.cell_factor == b.cell_factor &&
           a.block_warps == b.block_warps && a.keep_candidates == b.keep_candidates;
}

static void drop_graph(ac_ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_launches = 0;
}

// Capture the replay sequence (build_body with the recorded sizes and the
// device checks in place of the readbacks) as a graph, on the context's own
// stream; the graph is then launched on the caller's.
static int capture_replay(ac_ctx* c) {
    cudaStream_t s = c->cap_stream;
    c->expects.clear();
    AC_TRY(c->expect_table.reserve(MAX_EXPECTS * sizeof(ExpectEntry), s));
    AC_CUDA(cudaStreamSynchronize(s));
    AC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const long long l0 = g_launch_count;
    c->replaying = true;
    g_no_alloc = true;
    const int rc = build_body(c, s);
    g_no_alloc = false;
    c->replaying = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != AC_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != AC_OK ? rc : fail(AC_ERR_CUDA, "graph capture of the build failed");
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(AC_ERR_CUDA, "graph instantiation failed");
    }
    // the checks the graph runs: their table sits at a fixed address the graph captured
    if (!c->expects.empty() &&
        cudaMemcpy(c->expect_table.p, c->expects.data(), c->expects.size() * sizeof(ExpectEntry),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGraphExecDestroy(ex);
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(AC_ERR_CUDA, "upload of the replay checks failed");
    }
    c->graph = g;
    c->graph_exec = ex;
    c->graph_launches = g_launch_count - l0;
    return AC_OK;
}

// Sizes of a successful synchronised build, for the replays.
static int record_build(ac_ctx* c, const DevCounters& post, cudaStream_t s) {
    ac::BuildRecord& r = c->rec;
    r.opt = c->opt;
    r.wmax = (int)(c->pc.H2 - c->pc.A);
    r.nb_total = c->nb_total;
    r.nb_stride = c->nb_stride;
    r.n_wide = c->n_wide;
    r.n_huge = c->n_huge;
    r.n_w128 = c->n_w128;
    r.n_w256 = c->n_w256;
    r.post = post;
    r.post.err = 0;
    r.n_pending = (int64_t)post.n_pending;
    for (int d = 0; d < 4; d++) r.count[d] = c->K[d].count;
    for (int d = 1; d < 4; d++) r.count[3 + d] = c->C[d].count;
    r.valid = true;
    return AC_OK;
}

// The plan bounds a replay checks against, copied before the build's last host
// wait (which then also completes them, before a replay on another stream reads them).
static int record_copies(ac_ctx* c, cudaStream_t s) {
    const size_t nb = (size_t)c->n_mol * 6;
    AC_TRY(c->rec_bbox.reserve((nb + 1) * sizeof(int32_t), s));
    AC_CUDA(cudaMemcpyAsync(c->rec_bbox.p, c->scratch[0].p, nb * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    AC_CUDA(cudaMemcpyAsync(c->rec_bbox.as<int32_t>() + nb, c->scratch[1].p, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                            s));
    return AC_OK;
}

extern "C" int ac_build(ac_ctx* c, void* stream) {
    if (!c) return fail(AC_ERR_INVALID_ARG, "ctx is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    StreamScope scope(s);
    c->built = false;
    c->host_syncs = 0;
    const long long launches0 = g_launch_count;
    bool replayed = false;
    DevCounters h;
    if (c->rec.valid && !c->opt.no_graph && same_plan(c->rec.opt, c->opt)) {
        if (!c->graph_exec && capture_replay(c) != AC_OK) {
            drop_graph(c);
            c->rec.valid = false;
        }
        if (c->graph_exec) {
            AC_CUDA(cudaGraphLaunch(c->graph_exec, s));
            AC_TRY(read_counters(c, &h, s));
            if (h.err & (DERR_REPLAY | DERR_DEGREE)) {
                // a size moved (or a row outgrew the recorded masks): forget the graph and build with readbacks
                drop_graph(c);
                c->rec.valid = false;
                unsigned zero = 0;
                AC_CUDA(cudaMemcpy(&c->counters.as<DevCounters>()->err, &zero, sizeof(zero), cudaMemcpyHostToDevice));
            } else {
                replayed = true;
            }
        }
    }
    if (!replayed) {
        drop_graph(c);
        AC_TRY(build_body(c, s));
        if (!c->opt.no_graph) AC_TRY(record_copies(c, s));
        AC_TRY(read_counters(c, &h, s));
    }
    if (h.err & DERR_INTERNAL)
        return fail(AC_ERR_CUDA,
                    "internal invariant failed (an attached simplex without a coface, a simplex of K^1 or K^2 whose "
                    "vertices are not neighbours, or a K^3 row count that differs from the emitted tetrahedra)");
    if (h.err & DERR_TIMEOUT) {
        drop_graph(c);
        c->rec.valid = false;
        return fail(AC_ERR_TIMEOUT, "a bounded device wait (scan look-back) ran out");
    }
    if (!replayed && !c->opt.no_graph) AC_TRY(record_build(c, h, s));
    finish_mol_rows(c);
    const DevCounters& hl = h;  // the per-atom pass wrote them; later stages add only error bits
    ac_stats& st = c->stats;
    st.n_atoms = c->n;
    st.candidates[0] = 0;
    for (int d = 1; d < 4; d++) st.candidates[d] = (int64_t)hl.n_cand[d];
    for (int d = 0; d < 4; d++) st.simplices[d] = c->K[d].count;
    st.neighbour_pairs = c->nb_total;
    st.max_degree = hl.max_degree;
    for (int k = 0; k < 3; k++) {
        st.ac2_tests_tet[k] = (int64_t)hl.ac2_tet[k];
        st.ac2_tests_tri[k] = (int64_t)hl.ac2_tri[k];
    }
    st.ac2_tests_edge = (int64_t)hl.ac2_edge;
    for (int d = 0; d < 4; d++) st.ac3_tests[d] = (int64_t)hl.ac3[d];
    st.ac3_exact = (int64_t)hl.ac3_exact;
    st.escalated = (int64_t)hl.n_pending;
    st.ms_stage[0] = elapsed(c->ev[0], c->ev[1]);
    st.ms_stage[1] = elapsed(c->ev[1], c->ev[2]);
    st.ms_stage[2] = elapsed(c->ev[2], c->ev[3]);
    st.ms_stage[3] = elapsed(c->ev[3], c->ev[4]);
    st.ms_stage[4] = elapsed(c->ev[4], c->ev[5]);
    st.ms_stage[5] = elapsed(c->ev[5], c->ev[6]);
    st.ms_stage[6] = elapsed(c->ev[6], c->ev[7]);
    st.ms_stage[7] = c->n > 0 ? elapsed(c->ev[8], c->ev[9]) : 0.0;  // the per-atom kernels
    st.ms_total = elapsed(c->ev[0], c->ev[7]);
    st.kernel_launches = replayed ? c->graph_launches : g_launch_count - launches0;
    st.replayed = replayed ? 1 : 0;
    st.host_syncs = c->host_syncs;
    c->built = true;
    return AC_OK;
}

static int get_list(ac_ctx* c, ac::SimplexList* L, int dim, int64_t mol, int64_t* first, int64_t* count) {
    if (!c || dim < 0 || dim > 3 || !count) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!c->built) return fail(AC_ERR_STATE, "no successful ac_build on this context");
    int64_t m = mol < 0 ? 0 : mol;
    if (mol < -1 || m >= c->n_mol || (mol == -1 && c->n_mol != 1))
        return fail(AC_ERR_INVALID_ARG, "molecule index out of range");
    ac::SimplexList& S = L[dim];
    *first = S.mol_off.empty() ? 0 : S.mol_off[(size_t)m];
    *count = S.mol_off.empty() ? 0 : S.mol_off[(size_t)m + 1] - S.mol_off[(size_t)m];
    return AC_OK;
}

extern "C" int ac_get_simplices(ac_ctx* c, int dim, int64_t mol, const int32_t** d_tuples, int64_t* count) {
    int64_t first = 0;
    AC_TRY(get_list(c, c ? c->K : nullptr, dim, mol, &first, count));
    if (!d_tuples) return fail(AC_ERR_INVALID_ARG, "d_tuples is NULL");
    *d_tuples = c->K[dim].tuples.as<int32_t>() + first * (dim + 1);
    return AC_OK;
}

extern "C" int ac_filtration_values(ac_ctx* c, int dim, int64_t mol, const double** d_f, int64_t* count) {
    int64_t first = 0;
    AC_TRY(get_list(c, c ? c->K : nullptr, dim, mol, &first, count));
    if (!d_f) return fail(AC_ERR_INVALID_ARG, "d_f is NULL");
    const ac::DevBuf& b = c->opt.filtration == AC_FILTRATION_ORTHOSIZE ? c->K[dim].orthosize : c->K[dim].f;
    *d_f = b.as<double>() + first;
    return AC_OK;
}

extern "C" int ac_attached_flags(ac_ctx* c, int dim, int64_t mol, const uint8_t** d_flags, int64_t* count) {
    int64_t first = 0;
    AC_TRY(get_list(c, c ? c->K : nullptr, dim, mol, &first, count));
    if (!d_flags) return fail(AC_ERR_INVALID_ARG, "d_flags is NULL");
    *d_flags = c->K[dim].attached.as<uint8_t>() + first;
    return AC_OK;
}

extern "C" int ac_get_simplices_host(ac_ctx* c, int dim, int64_t mol, const int32_t** h_tuples, const double** h_f,
                                     const uint8_t** h_attached, int64_t* count) {
    int64_t first = 0;
    AC_TRY(get_list(c, c ? c->K : nullptr, dim, mol, &first, count));
    if (!c->opt.host_results) return fail(AC_ERR_STATE, "context does not keep host results (opt.host_results)");
    const int64_t total = c->K[dim].count;
    const int k = dim + 1;
    char* b = static_cast<char*>(c->hres[dim]);
    if (total > 0 && !b) return fail(AC_ERR_STATE, "no host copy of this list");
    if (h_tuples) *h_tuples = total > 0 ? reinterpret_cast<const int32_t*>(b) + first * k : nullptr;
    if (h_f) *h_f = total > 0 ? reinterpret_cast<const double*>(b + hres_f_off(total, k)) + first : nullptr;
    if (h_attached) *h_attached = total > 0 ? reinterpret_cast<const uint8_t*>(b + hres_a_off(total, k)) + first : nullptr;
    return AC_OK;
}

extern "C" int ac_get_candidates(ac_ctx* c, int dim, const int32_t** d_tuples, int64_t* count) {
    if (!c || dim < 1 || dim > 3 || !d_tuples || !count) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!c->built) return fail(AC_ERR_STATE, "no successful ac_build on this context");
    if (!c->opt.keep_candidates || c->n_mol != 1) return fail(AC_ERR_STATE, "context does not keep candidates");
    *d_tuples = c->C[dim].tuples.as<int32_t>();
    *count = c->C[dim].count;
    return AC_OK;
}

extern "C" int ac_eval_filtration(ac_ctx* c, const double* d_centres, const double* d_radii, double* const d_f_out[4],
                                  void* stream) {
    if (!c || !d_centres || !d_radii || !d_f_out) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!c->built) return fail(AC_ERR_STATE, "no successful ac_build on this context");
    StreamScope scope((cudaStream_t)stream);
    return eval_filtration(c, d_centres, d_radii, d_f_out, (cudaStream_t)stream);
}

extern "C" int ac_eval_filtration_fp32(ac_ctx* c, float* const d_f_out[4], void* stream) {
    if (!c || !d_f_out) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!c->built) return fail(AC_ERR_STATE, "no successful ac_build on this context");
    StreamScope scope((cudaStream_t)stream);
    return eval_filtration_f32(c, d_f_out, (cudaStream_t)stream);
}

extern "C" int ac_backward(ac_ctx* c, const double* const d_dLdf[4], double* d_dLdcentres, double* d_dLdradii,
                           void* stream) {
    if (!c || !d_dLdf || !d_dLdcentres || !d_dLdradii) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!c->built) return fail(AC_ERR_STATE, "no successful ac_build on this context");
    StreamScope scope((cudaStream_t)stream);
    return backward(c, d_dLdf, d_dLdcentres, d_dLdradii, (cudaStream_t)stream);
}

extern "C" int ac_backward_noalloc(ac_ctx* c, const double* const d_dLdf[4], double* d_dLdcentres,
                                   double* d_dLdradii, void* stream) {
    if (!c || !d_dLdf || !d_dLdcentres || !d_dLdradii) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!c->built) return fail(AC_ERR_STATE, "no successful ac_build on this context");
    return backward_noalloc(c, d_dLdf, d_dLdcentres, d_dLdradii, (cudaStream_t)stream);
}

extern "C" int ac_subcomplex(ac_ctx* c, int dim, int64_t mol, double alpha2, uint8_t* d_flags, int64_t* count_in,
                             void* stream) {
    int64_t first = 0, count = 0;
    AC_TRY(get_list(c, c ? c->K : nullptr, dim, mol, &first, &count));
    if (!count_in || (count > 0 && !d_flags)) return fail(AC_ERR_INVALID_ARG, "bad argument");
    if (!(alpha2 <= c->alpha)) return fail(AC_ERR_INVALID_ARG, "alpha2 must not exceed the context's alpha");
    if (!(alpha2 * 1048576.0 > -9.2e18)) return fail(AC_ERR_INVALID_ARG, "alpha2 out of range");
    StreamScope scope((cudaStream_t)stream);
    return subcomplex_flags(c, dim, first, count, alpha2, d_flags, count_in, (cudaStream_t)stream);
}

extern "C" int ac_autotune(ac_ctx* c, void* stream, ac_options* chosen) {
    if (!c) return fail(AC_ERR_INVALID_ARG, "ctx is NULL");
    c->plan_fresh = false;  // every trial plans its own grid
    // grid cell side (in units of h) and warps per block of the per-atom kernel
    // (cells below h pay off for inputs with widely spread radii, above h for sparse ones)
    const double factors[6] = {0.5, 0.75, 1.0, 1.25, 1.5, 2.0};
    const int warps[3] = {4, 6, 8};
    const ac_options base = c->opt;
    ac_options best = base;
    double best_ms = INFINITY;
    for (double f : factors)
        for (int w : warps) {
            c->opt = base;
            c->opt.cell_factor = f;
            c->opt.block_warps = w;
            double ms = 0.0;
            for (int rep = 0; rep < 2; rep++) {  // the first build of a shape also sizes its buffers
                AC_TRY(ac_build(c, stream));
                ms = c->stats.ms_total;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = c->opt;
            }
        }
    c->opt = best;
    AC_TRY(ac_build(c, stream));
    if (chosen) *chosen = best;
    return AC_OK;
}

extern "C" int ac_get_stats(ac_ctx* c, ac_stats* out) {
    if (!c || !out) return fail(AC_ERR_INVALID_ARG, "bad argument");
    *out = c->stats;
    return AC_OK;
}

extern "C" int ac_get_sizes(ac_ctx* c, int64_t* n_mol, int64_t* n_atoms) {
    if (!c) return fail(AC_ERR_INVALID_ARG, "ctx is NULL");
    if (n_mol) *n_mol = c->n_mol;
    if (n_atoms) *n_atoms = c->n;
    return AC_OK;
}

extern "C" void ac_destroy(ac_ctx* c) {
    if (!c) return;
    // the context's buffers go back to the pool once no work can still use them;
    // after a clean synchronisation they are idle and wait for the next context
    const bool idle = cudaDeviceSynchronize() == cudaSuccess;
    StreamScope scope(nullptr);
    struct IdleScope {
        explicit IdleScope(bool on) { g_release_idle = on; }
        ~IdleScope() { g_release_idle = false; }
    } idle_scope(idle);
    drop_graph(c);
    for (int d = 0; d < 4; d++) host_block_give(c->hres[d], c->hres_bytes[d]);
    CtxRes r;
    r.device = c->res_device;
    for (int k = 0; k < 10; k++) r.ev[k] = c->ev[k];
    r.ev_fork = c->ev_fork;
    r.ev_join = c->ev_join;
    r.ev_copy = c->ev_copy;
    r.ev_cjoin = c->ev_cjoin;
    r.side = c->side;
    r.copy = c->copy;
    r.cap_stream = c->cap_stream;
    r.pinned = c->h_pinned;
    r.pinned_bytes = c->h_pinned_bytes;
    // a set from a failed creation is incomplete: free it rather than cache it
    bool whole = r.device >= 0 && r.pinned && r.side && r.cap_stream && r.copy && r.ev_fork && r.ev_join &&
                 r.ev_copy && r.ev_cjoin;
    for (int k = 0; k < 10; k++) whole = whole && r.ev[k];
    if (whole && cudaGetLastError() == cudaSuccess) res_give(r);
    else res_free(r);
    delete c;
}

extern "C" const char* ac_error_string(int code) {
    switch (code) {
        case AC_OK: return "ok";
        case AC_ERR_INVALID_ARG: return "invalid argument";
        case AC_ERR_DEGENERATE: return "degenerate input (coincident centres)";
        case AC_ERR_RANGE: return "input outside the exact-integer range";
        case AC_ERR_CAPACITY: return "internal list capacity exceeded";
        case AC_ERR_OOM: return "out of device memory";
        case AC_ERR_CUDA: return "CUDA runtime error";
        case AC_ERR_TIMEOUT: return "bounded device wait timed out";
        case AC_ERR_STATE: return "no results: call ac_build first";
        default: return "unknown error";
    }
}

extern "C" const char* ac_last_error_detail(void) { return g_detail.c_str(); }
