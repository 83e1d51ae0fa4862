// ivs_clusters.cu -- root isolation and backtracking over a solve's accepted boxes (host).
//
// Section 3.4: the last round leaves many tiny configurations; merging them gives bigger,
// readable ones and isolates the real roots.  ivs_clusters merges boxes that touch into
// connected components (one per isolated root); ivs_backtrack counts the configurations
// of a coarser round that the boxes map to (Algorithm 5, read on the dyadic grid of the
// initial box), the count the paper tabulates per width.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "../../include/ivsolve.h"
#include "ivs_hostcore.h"

using namespace ivs::host;

namespace {

int64_t uf_find(std::vector<int64_t> &par, int64_t a) {
    int64_t r = a;
    while (par[r] != r) r = par[r];
    while (par[a] != r) {   // path compression
        const int64_t nx = par[a];
        par[a] = r;
        a = nx;
    }
    return r;
}

constexpr double kMaxPairTests = 4e9;

// Connected components of touching boxes: par[i] ends as the smallest box index of i's
// component.  False when the sweep would test more than kMaxPairTests pairs.
bool touch_components(int n, int64_t count, const double *lo, const double *hi, std::vector<int64_t> &par) {
    // sweep over the first coordinate: boxes in order of lo_0; a box can only touch the
    // boxes still open there (hi_0 >= its lo_0)
    std::vector<int64_t> order((size_t)count);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return lo[a * n] < lo[b * n]; });
    par.resize((size_t)count);
    std::iota(par.begin(), par.end(), (int64_t)0);
    std::vector<int64_t> open;
    double tests = 0;
    for (int64_t i : order) {
        const double l0 = lo[i * n];
        size_t keep = 0;
        for (size_t q = 0; q < open.size(); q++)
            if (hi[open[q] * n] >= l0) open[keep++] = open[q];
        open.resize(keep);
        tests += (double)open.size();
        if (tests > kMaxPairTests) return false;
        for (int64_t a : open) {
            bool touch = true;
            for (int j = 0; j < n && touch; j++) touch = lo[a * n + j] <= hi[i * n + j] && lo[i * n + j] <= hi[a * n + j];
            if (!touch) continue;
            const int64_t ra = uf_find(par, a), ri = uf_find(par, i);
            if (ra != ri) par[std::max(ra, ri)] = std::min(ra, ri);   // root = smallest box index
        }
        open.push_back(i);
    }
    for (int64_t i = 0; i < count; i++) par[(size_t)i] = uf_find(par, i);
    return true;
}

}  // namespace

extern "C" {

int ivs_clusters(int32_t n_vars, int64_t count, const double *lo, const double *hi, int64_t *n_clusters,
                 int64_t *label, double *cl_lo, double *cl_hi, int64_t cl_cap) {
    if (!n_clusters || n_vars <= 0 || n_vars > 16 || count < 0 || (count > 0 && (!lo || !hi)))
        return fail(IVS_ERR_INVALID, "ivs_clusters: bad arguments");
    *n_clusters = 0;
    if (count == 0) return IVS_OK;
    const int n = n_vars;
    std::vector<int64_t> par;
    if (!touch_components(n, count, lo, hi, par)) return fail(IVS_ERR_BUDGET, "ivs_clusters: too many overlapping boxes");
    // clusters numbered in the order of their first box
    std::vector<int64_t> num((size_t)count, -1);
    int64_t nc = 0;
    for (int64_t i = 0; i < count; i++) {
        const int64_t r = uf_find(par, i);
        if (num[r] < 0) num[r] = nc++;
        const int64_t c = num[r];
        if (label) label[i] = c;
        if (cl_lo && cl_hi && c < cl_cap) {
            for (int j = 0; j < n; j++) {
                const double a = lo[i * n + j], b = hi[i * n + j];
                if (num[r] == nc - 1 && r == i) {   // first box of this cluster
                    cl_lo[c * n + j] = a;
                    cl_hi[c * n + j] = b;
                } else {
                    cl_lo[c * n + j] = std::min(cl_lo[c * n + j], a);
                    cl_hi[c * n + j] = std::max(cl_hi[c * n + j], b);
                }
            }
        }
    }
    *n_clusters = nc;
    return IVS_OK;
}

int ivs_backtrack(int32_t n_vars, int64_t count, const double *lo, const double *hi, const double *box_lo,
                  const double *box_hi, int32_t level, int64_t max_cells, int64_t *n_cells, int64_t *n_groups) {
    if (!n_cells || n_vars <= 0 || n_vars > 16 || count < 0 || level < 0 || level > 30 || !box_lo || !box_hi ||
        (count > 0 && (!lo || !hi)))
        return fail(IVS_ERR_INVALID, "ivs_backtrack: bad arguments");
    *n_cells = 0;
    if (n_groups) *n_groups = 0;
    const int n = n_vars;
    const int64_t side = (int64_t)1 << level;
    std::vector<double> w((size_t)n);
    for (int j = 0; j < n; j++) {
        if (!(box_hi[j] > box_lo[j])) return fail(IVS_ERR_INVALID, "ivs_backtrack: empty initial box");
        w[(size_t)j] = std::ldexp(box_hi[j] - box_lo[j], -level);
    }
    std::vector<int32_t> cells;
    int32_t a[16], b[16], cur[16];
    int64_t total = 0;
    for (int64_t i = 0; i < count; i++) {
        int64_t m = 1;
        for (int j = 0; j < n; j++) {
            const double tl = (lo[i * n + j] - box_lo[j]) / w[(size_t)j];
            const double th = (hi[i * n + j] - box_lo[j]) / w[(size_t)j];
            const double fa = std::floor(tl), fb = std::ceil(th) - 1.0;
            double x = fa < fb ? fa : fb, y = fa < fb ? fb : fa;
            if (x < 0) x = 0;
            if (y > (double)(side - 1)) y = (double)(side - 1);
            if (y < x) y = x;   // a box outside the grid: the nearest cell
            if (x > (double)(side - 1)) x = y = (double)(side - 1);
            a[j] = (int32_t)x;
            b[j] = (int32_t)y;
            m *= (int64_t)(b[j] - a[j] + 1);
            if (m > max_cells) return fail(IVS_ERR_BUDGET, "ivs_backtrack: too many cells");
        }
        if (total + m > max_cells) return fail(IVS_ERR_BUDGET, "ivs_backtrack: too many cells");
        for (int j = 0; j < n; j++) cur[j] = a[j];
        for (int64_t q = 0; q < m; q++) {   // every cell of the box's index ranges
            cells.insert(cells.end(), cur, cur + n);
            total++;
            for (int j = 0; j < n; j++) {
                if (cur[j] < b[j]) {
                    cur[j]++;
                    break;
                }
                cur[j] = a[j];
            }
        }
    }
    std::vector<int64_t> idx((size_t)total);
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    auto less = [&](int64_t x, int64_t y) {
        return std::lexicographical_compare(cells.begin() + x * n, cells.begin() + (x + 1) * n, cells.begin() + y * n,
                                            cells.begin() + (y + 1) * n);
    };
    std::sort(idx.begin(), idx.end(), less);
    std::vector<double> ul, uh;   // the distinct cells as closed unit boxes of index space
    int64_t distinct = 0;
    for (int64_t q = 0; q < total; q++)
        if (q == 0 || std::memcmp(&cells[(size_t)(idx[q - 1] * n)], &cells[(size_t)(idx[q] * n)], sizeof(int32_t) * n) != 0) {
            distinct++;
            if (n_groups)
                for (int j = 0; j < n; j++) {
                    ul.push_back((double)cells[(size_t)(idx[q] * n + j)]);
                    uh.push_back((double)cells[(size_t)(idx[q] * n + j)] + 1.0);
                }
        }
    *n_cells = distinct;
    if (n_groups && distinct > 0) {
        // cells touch when their indices differ by at most 1 in every coordinate: union
        // each cell with the neighbours among the 3^n - 1 offsets that exist (hash lookup)
        double work = (double)distinct;
        for (int j = 0; j < n; j++) work *= 3.0;
        if (work > kMaxPairTests) return fail(IVS_ERR_BUDGET, "ivs_backtrack: too many cells to group");
        auto key_of = [&](const int32_t *c) {
            uint64_t h = 1469598103934665603ull;
            for (int j = 0; j < n; j++) h = (h ^ (uint64_t)(uint32_t)c[j]) * 1099511628211ull;
            return h;
        };
        std::vector<int32_t> uc((size_t)(distinct * n));
        for (int64_t q = 0; q < distinct; q++)
            for (int j = 0; j < n; j++) uc[(size_t)(q * n + j)] = (int32_t)ul[(size_t)(q * n + j)];
        std::unordered_map<uint64_t, std::vector<int64_t>> where;
        where.reserve((size_t)distinct * 2);
        for (int64_t q = 0; q < distinct; q++) where[key_of(&uc[(size_t)(q * n)])].push_back(q);
        std::vector<int64_t> par((size_t)distinct);
        std::iota(par.begin(), par.end(), (int64_t)0);
        int32_t nb[16], off[16];
        for (int64_t q = 0; q < distinct; q++) {
            const int32_t *c = &uc[(size_t)(q * n)];
            for (int j = 0; j < n; j++) off[j] = -1;
            for (;;) {
                bool zero = true;
                for (int j = 0; j < n; j++) {
                    nb[j] = c[j] + off[j];
                    zero = zero && off[j] == 0;
                }
                if (!zero) {
                    auto it = where.find(key_of(nb));
                    if (it != where.end())
                        for (int64_t o : it->second)
                            if (std::memcmp(&uc[(size_t)(o * n)], nb, sizeof(int32_t) * n) == 0) {
                                const int64_t ra = uf_find(par, q), rb = uf_find(par, o);
                                if (ra != rb) par[std::max(ra, rb)] = std::min(ra, rb);
                            }
                }
                int j = 0;   // next offset in {-1, 0, 1}^n
                while (j < n && off[j] == 1) off[j++] = -1;
                if (j == n) break;
                off[j]++;
            }
        }
        int64_t g = 0;
        for (int64_t q = 0; q < distinct; q++) g += uf_find(par, q) == q ? 1 : 0;
        *n_groups = g;
    }
    return IVS_OK;
}

}  // extern "C"
