// ivs_roots.cu -- root isolation and Algorithm 5 backtracking on the GPU.
//
// Section 3.4: the last round leaves many tiny configurations; merging them isolates the
// real roots.  Two device pipelines over a solve's accepted boxes (a plan's result region,
// or host rows copied in), with the same results as the host versions in ivs_clusters.cu:
//
// backtracking (Algorithm 5, read on the dyadic grid of the initial box): per box the cell
//   ranges of level L per coordinate (t = (x - d_lo) / w in round to nearest, cells
//   floor(t_lo) .. ceil(t_hi) - 1, swapped when they cross, clamped), a scan of the cell
//   counts, one 128-bit key per (box, cell) (coordinate 0 in the most significant bits),
//   a bitonic sort, unique -> the distinct cells; then the groups (connected components of
//   cells whose indices differ by at most 1 in every coordinate): in key order every
//   neighbour of a cell with a larger key has coordinate 0 at most one above, so each
//   cell tests the cells after it up to that bound (binary search) and unites with the
//   touching ones (lock-free union-find, roots = smallest index).
// clusters (connected components of touching boxes): boxes sorted by (lo_0, index); a box
//   can only touch the later boxes whose lo_0 <= its hi_0 (binary search), so each tests
//   those; clusters are numbered in the order of their first box (a scan over the
//   "first box of its component" flags) and their hulls taken with atomic min / max.
//
// Every loop that waits on other threads' progress (the union-find retry loop) has an
// iteration limit after which the kernel sets an error flag and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/ivsolve.h"
#include "ivs_hostcore.h"

using namespace ivs;
using namespace ivs::host;

// the plan's device-resident result region of one system (ivs_host.cu)
int plan_result_view(ivs_plan *p, int32_t s, const double **lo, const double **hi, int64_t *count, int64_t *stride,
                     int *n, const double **box_lo, const double **box_hi, cudaStream_t *st, int *device);

namespace {

constexpr double kMaxPairTests = 4e9;
constexpr int kUfIters = 1 << 20;   // retries of one union before the kernel gives up

// A set of boxes in device memory: coordinate j of box i at lo[i * rs + j * cs].
struct BoxView {
    const double *lo, *hi;
    int64_t rs, cs, count;
    int n;
    __device__ __forceinline__ double l(int64_t i, int j) const { return lo[i * rs + (int64_t)j * cs]; }
    __device__ __forceinline__ double h(int64_t i, int j) const { return hi[i * rs + (int64_t)j * cs]; }
};

struct Key {
    unsigned long long a, b;   // a: high word
};
__device__ __forceinline__ bool key_less(Key x, Key y) { return x.a < y.a || (x.a == y.a && x.b < y.b); }

// ---- scan (exclusive, int64) -------------------------------------------------------------
constexpr int kScanThreads = 1024;

__global__ void k_scan_blocks(const int64_t *in, int64_t *out, int64_t count, int64_t *sums) {
    __shared__ int64_t s[kScanThreads];
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kScanThreads + t;
    const int64_t v = i < count ? in[i] : 0;
    s[t] = v;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const int64_t x = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += x;
        __syncthreads();
    }
    if (i < count) out[i] = s[t] - v;
    if (t == kScanThreads - 1) sums[blockIdx.x] = s[t];
}

__global__ void k_scan_add(int64_t *out, int64_t count, const int64_t *offs) {
    const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
    if (i < count) out[i] += offs[blockIdx.x];
}

// exclusive scan of count values; *total (device) receives their sum
cudaError_t scan_exclusive(const int64_t *in, int64_t *out, int64_t count, int64_t *total, cudaStream_t st,
                           std::vector<void *> &scratch) {
    if (count <= 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), st);
    const int64_t nb = (count + kScanThreads - 1) / kScanThreads;
    int64_t *sums = nullptr, *offs = nullptr;
    cudaError_t e = cudaMalloc(&sums, (size_t)nb * sizeof(int64_t));
    if (e == cudaSuccess) scratch.push_back(sums);
    if (e == cudaSuccess) e = cudaMalloc(&offs, (size_t)nb * sizeof(int64_t));
    if (e == cudaSuccess) scratch.push_back(offs);
    if (e != cudaSuccess) return e;
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, count, sums);
    if (nb == 1) return cudaMemcpyAsync(total, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    e = scan_exclusive(sums, offs, nb, total, st, scratch);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, count, offs);
    return cudaGetLastError();
}

// ---- bitonic sort of 128-bit keys ----------------------------------------------------------
constexpr int kSortBlock = 1024;   // elements per shared-memory stage

__global__ void k_bitonic_global(Key *k, int64_t N, int64_t j, int64_t kk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t l = i ^ j;
    if (l <= i) return;
    const Key x = k[i], y = k[l];
    const bool up = (i & kk) == 0;
    if (up ? key_less(y, x) : key_less(x, y)) {
        k[i] = y;
        k[l] = x;
    }
}

// stages j = jmax .. 1 of merge size kk inside blocks of kSortBlock elements; with
// kk = 0 the whole sort of every block (kk = 2 .. kSortBlock)
__global__ void k_bitonic_shared(Key *k, int64_t N, int64_t kk, int64_t jmax) {
    __shared__ Key s[kSortBlock];
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
    for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) s[t] = k[base + t];
    __syncthreads();
    const int64_t k0 = kk ? kk : 2, k1 = kk ? kk : kSortBlock;
    for (int64_t q = k0; q <= k1; q <<= 1) {
        for (int64_t j = kk ? jmax : q / 2; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) {
                const int l = t ^ (int)j;
                if (l > t) {
                    const Key x = s[t], y = s[l];
                    const bool up = ((base + t) & q) == 0;
                    if (up ? key_less(y, x) : key_less(x, y)) {
                        s[t] = y;
                        s[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < kSortBlock; t += blockDim.x) k[base + t] = s[t];
}

// sorts N keys (N a power of two >= kSortBlock) ascending
cudaError_t bitonic_sort(Key *k, int64_t N, cudaStream_t st) {
    const unsigned blocks = (unsigned)(N / kSortBlock);
    k_bitonic_shared<<<blocks, 512, 0, st>>>(k, N, 0, 0);
    for (int64_t kk = 2 * kSortBlock; kk <= N; kk <<= 1) {
        int64_t j = kk / 2;
        for (; j >= kSortBlock; j >>= 1)
            k_bitonic_global<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(k, N, j, kk);
        k_bitonic_shared<<<blocks, 512, 0, st>>>(k, N, kk, j);
    }
    return cudaGetLastError();
}

__global__ void k_fill_keys(Key *k, int64_t from, int64_t to) {
    for (int64_t i = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < to; i += (int64_t)gridDim.x * blockDim.x)
        k[i] = Key{~0ull, ~0ull};
}

// ---- union-find -----------------------------------------------------------------------------
__device__ __forceinline__ int64_t uf_find(int64_t *par, int64_t x) {
    for (int it = 0; it < kUfIters; it++) {
        const int64_t p = par[x];
        if (p == x) return x;
        const int64_t gp = par[p];
        if (gp != p) atomicCAS((unsigned long long *)&par[x], (unsigned long long)p, (unsigned long long)gp);
        x = p;
    }
    return -1;
}

// unites the sets of a and b; the root with the larger index is hooked under the smaller
__device__ __forceinline__ bool uf_union(int64_t *par, int64_t a, int64_t b) {
    for (int it = 0; it < kUfIters; it++) {
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a < 0 || b < 0) return false;
        if (a == b) return true;
        if (a < b) {
            const int64_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS((unsigned long long *)&par[a], (unsigned long long)a, (unsigned long long)b) ==
            (unsigned long long)a)
            return true;
    }
    return false;
}

__global__ void k_iota(int64_t *par, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        par[i] = i;
}

// full compression; roots[i] = 1 when i is a root
__global__ void k_uf_flatten(int64_t *par, int64_t count, int64_t *is_root, int *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = uf_find(par, i);
        if (r < 0) {
            atomicExch(err, 1);
            continue;
        }
        par[i] = r;
        if (is_root) is_root[i] = r == i ? 1 : 0;
    }
}

// ---- backtracking kernels -------------------------------------------------------------------
struct Grid {
    double d_lo[kMaxVars], w[kMaxVars];
    int64_t side;
    int level, bits;   // bits = n * level (<= 127)
};

// cell index range of box i in coordinate j (the host rule, operation for operation)
__device__ __forceinline__ void cell_range(const BoxView &v, const Grid &g, int64_t i, int j, int32_t &a, int32_t &b) {
    const double tl = __ddiv_rn(__dsub_rn(v.l(i, j), g.d_lo[j]), g.w[j]);
    const double th = __ddiv_rn(__dsub_rn(v.h(i, j), g.d_lo[j]), g.w[j]);
    const double fa = floor(tl), fb = __dsub_rn(ceil(th), 1.0);
    double x = fa < fb ? fa : fb, y = fa < fb ? fb : fa;
    const double top = (double)(g.side - 1);
    if (x < 0) x = 0;
    if (y > top) y = top;
    if (y < x) y = x;
    if (x > top) x = y = top;
    a = (int32_t)x;
    b = (int32_t)y;
}

__global__ void k_bt_count(BoxView v, Grid g, int64_t max_cells, int64_t *m, int *over) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v.count; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 1;
        for (int j = 0; j < v.n; j++) {
            int32_t a, b;
            cell_range(v, g, i, j, a, b);
            c *= (int64_t)(b - a + 1);
            if (c > max_cells) {
                atomicExch(over, 1);
                c = 0;
                break;
            }
        }
        m[i] = c;
    }
}

// places field value c of coordinate j into the key (coordinate 0 most significant)
__device__ __forceinline__ void key_put(Key &k, const Grid &g, int n, int j, uint64_t c) {
    const int lsb = (n - 1 - j) * g.level;   // bit position of the field's lowest bit
    if (lsb >= 64) {
        k.a |= c << (lsb - 64);
    } else {
        k.b |= c << lsb;
        if (lsb + g.level > 64 && lsb > 0) k.a |= c >> (64 - lsb);
    }
}
__device__ __forceinline__ int32_t key_get(Key k, const Grid &g, int n, int j) {
    const int lsb = (n - 1 - j) * g.level;
    const uint64_t mask = (g.level >= 64) ? ~0ull : ((1ull << g.level) - 1ull);
    uint64_t v;
    if (lsb >= 64) v = k.a >> (lsb - 64);
    else if (lsb == 0) v = k.b;
    else v = (k.b >> lsb) | (k.a << (64 - lsb));
    return (int32_t)(v & mask);
}

__global__ void k_bt_emit(BoxView v, Grid g, const int64_t *offs, Key *keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v.count; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t a[kMaxVars], b[kMaxVars], cur[kMaxVars];
        int64_t m = 1;
        for (int j = 0; j < v.n; j++) {
            cell_range(v, g, i, j, a[j], b[j]);
            cur[j] = a[j];
            m *= (int64_t)(b[j] - a[j] + 1);
        }
        int64_t o = offs[i];
        for (int64_t q = 0; q < m; q++) {
            Key k{0ull, 0ull};
            for (int j = 0; j < v.n; j++) key_put(k, g, v.n, j, (uint64_t)cur[j]);
            keys[o + q] = k;
            for (int j = 0; j < v.n; j++) {   // next cell of the box's ranges
                if (cur[j] < b[j]) {
                    cur[j]++;
                    break;
                }
                cur[j] = a[j];
            }
        }
    }
}

__global__ void k_flag_distinct(const Key *k, int64_t total, int64_t *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || k[i].a != k[i - 1].a || k[i].b != k[i - 1].b) ? 1 : 0;
}

__global__ void k_compact(const Key *k, int64_t total, const int64_t *flag, const int64_t *pos, Key *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = k[i];
}

// first position in [lo, hi) whose key is >= x
__device__ __forceinline__ int64_t lower_bound(const Key *k, int64_t lo, int64_t hi, Key x) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (key_less(k[mid], x)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// the key just above every cell whose coordinate 0 is c0 + 1 (c0 + 2 in field 0, rest 0)
__device__ __forceinline__ Key field0_bound(const Grid &g, int n, int32_t c0) {
    Key k{0ull, 0ull};
    const uint64_t c = (uint64_t)c0 + 2ull;
    if (c >= (1ull << g.level)) return Key{~0ull, ~0ull};
    key_put(k, g, n, 0, c);
    return k;
}

// candidates of each distinct cell: the cells after it up to coordinate 0 + 1
__global__ void k_bt_ranges(const Key *u, int64_t d, Grid g, int n, int64_t *end, int64_t *work) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < d; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c0 = key_get(u[p], g, n, 0);
        const int64_t e = lower_bound(u, p + 1, d, field0_bound(g, n, c0));
        end[p] = e;
        work[p] = e - p - 1;
    }
}

// one warp per cell: unite it with the candidates whose indices differ by <= 1 everywhere
__global__ void k_bt_unite(const Key *u, int64_t d, Grid g, int n, const int64_t *end, int64_t *par, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < d; p += warps) {
        int32_t c[kMaxVars];
        for (int j = 0; j < n; j++) c[j] = key_get(u[p], g, n, j);
        for (int64_t q = p + 1 + lane; q < end[p]; q += 32) {
            bool touch = true;
            for (int j = 0; j < n && touch; j++) {
                const int32_t x = key_get(u[q], g, n, j);
                touch = x - c[j] <= 1 && c[j] - x <= 1;
            }
            if (touch && !uf_union(par, p, q)) atomicExch(err, 1);
        }
    }
}

__global__ void k_sum(const int64_t *v, int64_t count, unsigned long long *out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)v[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// ---- cluster kernels ---------------------------------------------------------------------------
// ordered integer image of a double (numeric order; -0 and +0 map to the same value)
__device__ __forceinline__ unsigned long long dkey(double x) {
    if (x == 0.0) x = 0.0;
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    const unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    return __longlong_as_double((long long)u);
}

__global__ void k_cl_keys(BoxView v, Key *k) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v.count; i += (int64_t)gridDim.x * blockDim.x)
        k[i] = Key{dkey(v.l(i, 0)), (unsigned long long)i};
}

// candidates of the box at sorted position p: the later positions with lo_0 <= its hi_0
__global__ void k_cl_ranges(BoxView v, const Key *k, int64_t *end, int64_t *work) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < v.count; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)k[p].b;
        const Key bound{dkey(v.h(i, 0)), ~0ull};
        int64_t lo = p + 1, hi = v.count;   // first position with key > (hi_0, any index)
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (!key_less(bound, k[mid])) lo = mid + 1;
            else hi = mid;
        }
        end[p] = lo;
        work[p] = lo - p - 1;
    }
}

__global__ void k_cl_unite(BoxView v, const Key *k, const int64_t *end, int64_t *par, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < v.count; p += warps) {
        const int64_t i = (int64_t)k[p].b;
        for (int64_t q = p + 1 + lane; q < end[p]; q += 32) {
            const int64_t o = (int64_t)k[q].b;
            bool touch = true;
            for (int j = 0; j < v.n && touch; j++) touch = v.l(o, j) <= v.h(i, j) && v.l(i, j) <= v.h(o, j);
            if (touch && !uf_union(par, i, o)) atomicExch(err, 1);
        }
    }
}

// first[i] = 1 when box i is the smallest index of its component (par[i] is its root, and
// the root is the smallest index: unions hook larger roots under smaller ones)
__global__ void k_cl_first(const int64_t *par, int64_t count, int64_t *first) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        first[i] = par[i] == i ? 1 : 0;
}

__global__ void k_cl_label(BoxView v, const int64_t *par, const int64_t *num, int64_t *label, int64_t cl_cap,
                           unsigned long long *hlo, unsigned long long *hhi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v.count; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = num[par[i]];
        label[i] = c;
        if (c < cl_cap)
            for (int j = 0; j < v.n; j++) {
                atomicMin(&hlo[c * v.n + j], dkey(v.l(i, j)));
                atomicMax(&hhi[c * v.n + j], dkey(v.h(i, j)));
            }
    }
}

__global__ void k_cl_hull_init(unsigned long long *hlo, unsigned long long *hhi, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        hlo[i] = ~0ull;
        hhi[i] = 0ull;
    }
}

__global__ void k_cl_hull_out(const unsigned long long *hlo, const unsigned long long *hhi, int64_t m, double *lo,
                              double *hi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        lo[i] = dkey_inv(hlo[i]);
        hi[i] = dkey_inv(hhi[i]);
    }
}

// ---- host drivers -----------------------------------------------------------------------------
struct Scratch {
    std::vector<void *> v;
    ~Scratch() {
        for (void *p : v) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T **p, size_t n) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) v.push_back(q);
        *p = (T *)q;
        return e;
    }
};

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

#define RT_TRY(x)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (x);                                                                       \
        if (e_ != cudaSuccess) return fail(IVS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int64_t pow2_at_least(int64_t x) {
    int64_t p = kSortBlock;
    while (p < x) p <<= 1;
    return p;
}

int backtrack_device(const BoxView &v, const double *box_lo, const double *box_hi, int32_t level, int64_t max_cells,
                     int64_t *n_cells, int64_t *n_groups, cudaStream_t st) {
    *n_cells = 0;
    if (n_groups) *n_groups = 0;
    const int n = v.n;
    if (level < 0 || level > 30) return fail(IVS_ERR_INVALID, "ivs_backtrack: level must be in 0..30");
    if ((int64_t)n * level > 127) return fail(IVS_ERR_INVALID, "backtracking on the GPU: n_vars * level must be <= 127");
    Grid g{};
    for (int j = 0; j < n; j++) {
        if (!(box_hi[j] > box_lo[j])) return fail(IVS_ERR_INVALID, "ivs_backtrack: empty initial box");
        g.d_lo[j] = box_lo[j];
        g.w[j] = std::ldexp(box_hi[j] - box_lo[j], -level);
    }
    g.side = (int64_t)1 << level;
    g.level = level;
    g.bits = n * level;
    if (v.count == 0) return IVS_OK;
    Scratch sc;
    int64_t *m = nullptr, *offs = nullptr, *tot = nullptr;
    int *flags = nullptr;   // [0] over budget, [1] union-find gave up
    RT_TRY(sc.get(&m, v.count));
    RT_TRY(sc.get(&offs, v.count));
    RT_TRY(sc.get(&tot, 2));
    RT_TRY(sc.get(&flags, 2));
    RT_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
    k_bt_count<<<grid_for(v.count), 256, 0, st>>>(v, g, max_cells, m, flags);
    RT_TRY(cudaGetLastError());
    RT_TRY(scan_exclusive(m, offs, v.count, tot, st, sc.v));
    int64_t total = 0;
    int hf[2] = {0, 0};
    RT_TRY(cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaStreamSynchronize(st));
    if (hf[0] || total > max_cells) return fail(IVS_ERR_BUDGET, "ivs_backtrack: too many cells");
    const int64_t N = pow2_at_least(total);
    Key *keys = nullptr, *uniq = nullptr;
    int64_t *fl = nullptr, *pos = nullptr;
    RT_TRY(sc.get(&keys, N));
    k_bt_emit<<<grid_for(v.count), 128, 0, st>>>(v, g, offs, keys);
    k_fill_keys<<<grid_for(N - total), 256, 0, st>>>(keys, total, N);
    RT_TRY(cudaGetLastError());
    RT_TRY(bitonic_sort(keys, N, st));
    RT_TRY(sc.get(&fl, total));
    RT_TRY(sc.get(&pos, total));
    k_flag_distinct<<<grid_for(total), 256, 0, st>>>(keys, total, fl);
    RT_TRY(scan_exclusive(fl, pos, total, tot, st, sc.v));
    int64_t d = 0;
    RT_TRY(cudaMemcpyAsync(&d, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RT_TRY(sc.get(&uniq, total));
    k_compact<<<grid_for(total), 256, 0, st>>>(keys, total, fl, pos, uniq);
    RT_TRY(cudaGetLastError());
    RT_TRY(cudaStreamSynchronize(st));
    *n_cells = d;
    if (!n_groups || d == 0) return IVS_OK;
    int64_t *end = nullptr, *work = nullptr, *par = nullptr;
    unsigned long long *wsum = nullptr;
    RT_TRY(sc.get(&end, d));
    RT_TRY(sc.get(&work, d));
    RT_TRY(sc.get(&par, d));
    RT_TRY(sc.get(&wsum, 1));
    RT_TRY(cudaMemsetAsync(wsum, 0, sizeof(unsigned long long), st));
    k_bt_ranges<<<grid_for(d), 256, 0, st>>>(uniq, d, g, n, end, work);
    k_sum<<<grid_for(d), 256, 0, st>>>(work, d, wsum);
    unsigned long long hw = 0;
    RT_TRY(cudaMemcpyAsync(&hw, wsum, sizeof(hw), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaStreamSynchronize(st));
    if ((double)hw > kMaxPairTests) return fail(IVS_ERR_BUDGET, "ivs_backtrack: too many cells to group");
    k_iota<<<grid_for(d), 256, 0, st>>>(par, d);
    k_bt_unite<<<grid_for(d * 32), 256, 0, st>>>(uniq, d, g, n, end, par, flags + 1);
    int64_t *root = work;   // reused
    k_uf_flatten<<<grid_for(d), 256, 0, st>>>(par, d, root, flags + 1);
    RT_TRY(cudaGetLastError());
    RT_TRY(cudaMemsetAsync(wsum, 0, sizeof(unsigned long long), st));
    k_sum<<<grid_for(d), 256, 0, st>>>(root, d, wsum);
    RT_TRY(cudaMemcpyAsync(&hw, wsum, sizeof(hw), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaStreamSynchronize(st));
    if (hf[1]) return fail(IVS_ERR_CUDA, "ivs_backtrack: union-find did not settle");
    *n_groups = (int64_t)hw;
    return IVS_OK;
}

int clusters_device(const BoxView &v, int64_t *n_clusters, int64_t *label_h, double *cl_lo, double *cl_hi,
                    int64_t cl_cap, cudaStream_t st) {
    *n_clusters = 0;
    if (v.count == 0) return IVS_OK;
    Scratch sc;
    const int64_t N = pow2_at_least(v.count);
    Key *keys = nullptr;
    int64_t *end = nullptr, *work = nullptr, *par = nullptr, *num = nullptr, *tot = nullptr, *label = nullptr;
    unsigned long long *wsum = nullptr, *hlo = nullptr, *hhi = nullptr;
    int *err = nullptr;
    RT_TRY(sc.get(&keys, N));
    RT_TRY(sc.get(&end, v.count));
    RT_TRY(sc.get(&work, v.count));
    RT_TRY(sc.get(&par, v.count));
    RT_TRY(sc.get(&wsum, 1));
    RT_TRY(sc.get(&err, 1));
    RT_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    RT_TRY(cudaMemsetAsync(wsum, 0, sizeof(unsigned long long), st));
    k_cl_keys<<<grid_for(v.count), 256, 0, st>>>(v, keys);
    k_fill_keys<<<grid_for(N - v.count), 256, 0, st>>>(keys, v.count, N);
    RT_TRY(cudaGetLastError());
    RT_TRY(bitonic_sort(keys, N, st));
    k_cl_ranges<<<grid_for(v.count), 256, 0, st>>>(v, keys, end, work);
    k_sum<<<grid_for(v.count), 256, 0, st>>>(work, v.count, wsum);
    unsigned long long hw = 0;
    RT_TRY(cudaMemcpyAsync(&hw, wsum, sizeof(hw), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaStreamSynchronize(st));
    if ((double)hw > kMaxPairTests) return fail(IVS_ERR_BUDGET, "ivs_clusters: too many overlapping boxes");
    k_iota<<<grid_for(v.count), 256, 0, st>>>(par, v.count);
    k_cl_unite<<<grid_for(v.count * 32), 256, 0, st>>>(v, keys, end, par, err);
    k_uf_flatten<<<grid_for(v.count), 256, 0, st>>>(par, v.count, nullptr, err);
    // clusters numbered in the order of their first box
    RT_TRY(sc.get(&num, v.count));
    RT_TRY(sc.get(&tot, 1));
    k_cl_first<<<grid_for(v.count), 256, 0, st>>>(par, v.count, work);
    RT_TRY(scan_exclusive(work, num, v.count, tot, st, sc.v));
    int64_t nc = 0;
    int he = 0;
    RT_TRY(cudaMemcpyAsync(&nc, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaMemcpyAsync(&he, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RT_TRY(cudaStreamSynchronize(st));
    if (he) return fail(IVS_ERR_CUDA, "ivs_clusters: union-find did not settle");
    *n_clusters = nc;
    if (!label_h && !(cl_lo && cl_hi && cl_cap > 0)) return IVS_OK;
    const int64_t cap = (cl_lo && cl_hi) ? std::min<int64_t>(cl_cap, nc) : 0;
    RT_TRY(sc.get(&label, v.count));
    RT_TRY(sc.get(&hlo, std::max<int64_t>(cap * v.n, 1)));
    RT_TRY(sc.get(&hhi, std::max<int64_t>(cap * v.n, 1)));
    k_cl_hull_init<<<grid_for(cap * v.n), 256, 0, st>>>(hlo, hhi, cap * v.n);
    k_cl_label<<<grid_for(v.count), 256, 0, st>>>(v, par, num, label, cap, hlo, hhi);
    RT_TRY(cudaGetLastError());
    if (label_h) RT_TRY(cudaMemcpyAsync(label_h, label, (size_t)v.count * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (cap > 0) {
        double *dl = (double *)end, *dh = (double *)work;   // reused (count >= cap * n? not always)
        if (cap * v.n > v.count) {
            RT_TRY(sc.get(&dl, cap * v.n));
            RT_TRY(sc.get(&dh, cap * v.n));
        }
        k_cl_hull_out<<<grid_for(cap * v.n), 256, 0, st>>>(hlo, hhi, cap * v.n, dl, dh);
        RT_TRY(cudaMemcpyAsync(cl_lo, dl, (size_t)(cap * v.n) * sizeof(double), cudaMemcpyDeviceToHost, st));
        RT_TRY(cudaMemcpyAsync(cl_hi, dh, (size_t)(cap * v.n) * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    RT_TRY(cudaStreamSynchronize(st));
    return IVS_OK;
}

// host rows (count x n, row-major) copied to the device
int upload_rows(Scratch &sc, int n, int64_t count, const double *lo, const double *hi, BoxView *v, cudaStream_t st) {
    double *dl = nullptr, *dh = nullptr;
    RT_TRY(sc.get(&dl, (size_t)count * n));
    RT_TRY(sc.get(&dh, (size_t)count * n));
    if (count > 0) {
        RT_TRY(cudaMemcpyAsync(dl, lo, (size_t)count * n * sizeof(double), cudaMemcpyHostToDevice, st));
        RT_TRY(cudaMemcpyAsync(dh, hi, (size_t)count * n * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    *v = BoxView{dl, dh, n, 1, count, n};
    return IVS_OK;
}

}  // namespace

extern "C" {

int ivs_clusters_gpu(int32_t n_vars, int64_t count, const double *lo, const double *hi, int64_t *n_clusters,
                     int64_t *label, double *cl_lo, double *cl_hi, int64_t cl_cap, int32_t device) {
    if (!n_clusters || n_vars <= 0 || n_vars > kMaxVars || count < 0 || (count > 0 && (!lo || !hi)))
        return fail(IVS_ERR_INVALID, "ivs_clusters_gpu: bad arguments");
    *n_clusters = 0;
    RT_TRY(cudaSetDevice(device));
    cudaStream_t st = nullptr;
    RT_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc;
    {
        Scratch sc;
        BoxView v{};
        rc = upload_rows(sc, n_vars, count, lo, hi, &v, st);
        if (rc == IVS_OK) rc = clusters_device(v, n_clusters, label, cl_lo, cl_hi, cl_cap, st);
        cudaStreamSynchronize(st);
    }
    cudaStreamDestroy(st);
    return rc;
}

int ivs_backtrack_gpu(int32_t n_vars, int64_t count, const double *lo, const double *hi, const double *box_lo,
                      const double *box_hi, int32_t level, int64_t max_cells, int64_t *n_cells, int64_t *n_groups,
                      int32_t device) {
    if (!n_cells || n_vars <= 0 || n_vars > kMaxVars || count < 0 || !box_lo || !box_hi ||
        (count > 0 && (!lo || !hi)))
        return fail(IVS_ERR_INVALID, "ivs_backtrack_gpu: bad arguments");
    *n_cells = 0;
    if (n_groups) *n_groups = 0;
    RT_TRY(cudaSetDevice(device));
    cudaStream_t st = nullptr;
    RT_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc;
    {
        Scratch sc;
        BoxView v{};
        rc = upload_rows(sc, n_vars, count, lo, hi, &v, st);
        if (rc == IVS_OK) rc = backtrack_device(v, box_lo, box_hi, level, max_cells, n_cells, n_groups, st);
        cudaStreamSynchronize(st);
    }
    cudaStreamDestroy(st);
    return rc;
}

int ivs_plan_backtrack(ivs_plan *p, int32_t s, int32_t level, int64_t max_cells, int64_t *n_cells,
                       int64_t *n_groups) {
    if (!p || !n_cells) return fail(IVS_ERR_INVALID, "ivs_plan_backtrack: bad arguments");
    const double *lo, *hi, *blo, *bhi;
    int64_t count, stride;
    int n, dev;
    cudaStream_t st;
    int rc = plan_result_view(p, s, &lo, &hi, &count, &stride, &n, &blo, &bhi, &st, &dev);
    if (rc) return rc;
    RT_TRY(cudaSetDevice(dev));
    BoxView v{lo, hi, 1, stride, count, n};
    return backtrack_device(v, blo, bhi, level, max_cells, n_cells, n_groups, st);
}

int ivs_plan_clusters(ivs_plan *p, int32_t s, int64_t *n_clusters) {
    if (!p || !n_clusters) return fail(IVS_ERR_INVALID, "ivs_plan_clusters: bad arguments");
    const double *lo, *hi, *blo, *bhi;
    int64_t count, stride;
    int n, dev;
    cudaStream_t st;
    int rc = plan_result_view(p, s, &lo, &hi, &count, &stride, &n, &blo, &bhi, &st, &dev);
    if (rc) return rc;
    RT_TRY(cudaSetDevice(dev));
    BoxView v{lo, hi, 1, stride, count, n};
    return clusters_device(v, n_clusters, nullptr, nullptr, nullptr, 0, st);
}

}  // extern "C"
