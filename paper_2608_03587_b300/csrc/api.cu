// C ABI of libdecbpm: mesh handles, plans, propagation and diagnostics.
// See include/decbpm.h for the contract of every entry point.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "decbpm.h"
#include "internal.h"
#include "kernels.cuh"

namespace decbpm {
const char *last_error_cstr();
}
using namespace decbpm;

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? DECBPM_ERR_OOM : DECBPM_ERR_CUDA,            \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);          \
        }                                                                                              \
    } while (0)

#define TRY(call)                        \
    do {                                 \
        int rc_ = (call);                \
        if (rc_ != DECBPM_OK) return rc_; \
    } while (0)

namespace {

// NVTX range around a public entry point (named in profiler timelines; a
// no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Tile maps of a mesh for one tile geometry (see build_tiles).
struct TileMaps {
    bool ready = false, ok = false;
    uint16_t *lcol = nullptr;
    int32_t *tdesc = nullptr, *halo_rows = nullptr, *halo_ovf = nullptr;
    int n_tiles = 0, max_halo = 0, max_entries = 0;
    // dataflow march: per tile kDepInts int32 (count, then the tiles adjacent
    // to it in the operator graph and itself); flow_ok if every list fits
    int32_t *tdeps = nullptr;
    bool flow_ok = false;
};

struct DevAllocs {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    template <class T> int alloc(T **p, size_t n) {
        *p = nullptr;
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
        if (e != cudaSuccess) {
            *p = nullptr;
            return fail(DECBPM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
        }
        ptrs.push_back((void *)*p);
        bytes += n * sizeof(T);
        return DECBPM_OK;
    }
    template <class T> int upload(T **p, const std::vector<T> &h) {
        TRY(alloc(p, h.size()));
        CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
        return DECBPM_OK;
    }
    void release() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
        bytes = 0;
    }
};

template <typename R> std::vector<R> cast(const std::vector<double> &x) { return std::vector<R>(x.begin(), x.end()); }

int ilog2(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

}  // namespace

// ============================================================== mesh handle
struct decbpm_mesh_s {
    Assembly A;
    Sell S;
    int device = 0;
    DevAllocs mem;
    int32_t *slice_ptr = nullptr, *slice_w = nullptr, *col = nullptr, *perm = nullptr;
    float *x32, *v32, *chib32, *sig32, *coff32, *cdiag32;
    double *x64, *v64, *chib64, *sig64, *coff64, *cdiag64, *w64, *m64;
    double *vbase64 = nullptr;   // base potential (internal order) that decbpm_mesh_set_potential_offset adds to
    int32_t *csr_ptr = nullptr, *csr_col = nullptr;
    double *csr_val = nullptr;
    std::map<std::pair<int, int>, decbpm_plan_t> plans;   // (fields, precision) -> cached single-mesh plan
    // geometry and materials in caller order, kept for operators assembled later (PML)
    std::vector<double> g_coords, g_V, g_chi;
    std::vector<int32_t> g_cells;
    // PML (complex-stretched metric): SELL weights a_pq = -K~_pq / m~_p and lumped v, chib
    bool pml_on = false;
    double2 *pml_a = nullptr, *pml_v = nullptr, *pml_chib = nullptr;
    // Gershgorin region of A~ (the union of the discs |z - sum_q a_pq| <= sum_q |a_pq|) as a box
    double pml_re_lo = 0, pml_re_hi = 0, pml_im_lo = 0, pml_im_hi = 0;
    // the split-step's scaled weights x_pq = a_pq / r (r, c: half width and
    // centre of the box's real extent) in both precisions, and v, chib in FP32
    double2 *pml_x64 = nullptr;
    float2 *pml_x32 = nullptr, *pml_v32 = nullptr, *pml_chib32 = nullptr;
    // tile maps of the tile-staged march (built on first use): 128-row tiles
    // of 16 fields (t16) and 512-row tiles of one field (t1)
    TileMaps t16, t1;
    // stage-pair maps (built on first use): per tile the depth-two halo list,
    // descriptor, and the SELL entries of the first halo ring
    bool pairs_ready = false, pairs_ok = false;
    int32_t *pdesc = nullptr, *hlist = nullptr;
    uint16_t *lcol2 = nullptr;
    float *x2 = nullptr;
    int max_nh1 = 0, max_nh12 = 0, max_hentries = 0;
    double r() const { return 0.5 * A.rho; }
};

// Per tile (128 rows of 16 fields, or with one = true 512 rows of one
// field): the sorted rows outside the tile that its SELL entries reference
// (halo; the first 96 at rows [96 t, 96 t + 96) of a padded list, the rest in
// an overflow list), for every entry its row in the tile's window (tile rows,
// then halo rows), and a descriptor of 8 int32:
//   {e0, ne, ovf, nh, es0 | es1 << 16, es2 | es3 << 16, w0 | w1 << 8 | w2 << 16 | w3 << 24, 0}
// (first entry and entry count, overflow offset and halo length, per-slice
// entry offsets relative to e0 and widths; the 512-row tiles leave the slice
// fields 0: their kernel copies the 16 slices' offsets and widths).  An
// entry's window row is stored as its byte offset (row * 128 for 16
// complex64 fields, row * 8 for one), so windows are limited to 511 or 8191
// rows; meshes with larger halos keep the row kernel.  Padding entries point
// inside the tile, so every window row a kernel reads was copied in.
static int build_tiles(decbpm_mesh_t M, bool one = false) {
    TileMaps &T = one ? M->t1 : M->t16;
    if (T.ready) return DECBPM_OK;
    const Sell &S = M->S;
    const int64_t n0 = M->A.n0;
    const int tile_rows = one ? kTile1Rows : kTileRows, row_bytes = one ? 8 : 128;
    const int nt = int((n0 + tile_rows - 1) / tile_rows);
    const int spt = tile_rows / kSlice;
    constexpr int held = 32 * kHaloRegs;                 // halo rows per tile at a fixed place
    std::vector<uint16_t> lcol(S.col.size(), 0);
    std::vector<int32_t> desc(size_t(nt) * 8, 0), hfixed(size_t(nt) * held, 0), hovf;
    std::vector<int32_t> uniq;
    std::vector<std::vector<int32_t>> adj(nt);          // tiles holding a tile's halo rows
    int max_halo = 0, max_entries = 0;
    for (int t = 0; t < nt; ++t) {
        const int64_t r0 = int64_t(t) * tile_rows, r1 = std::min<int64_t>(r0 + tile_rows, n0);
        const int64_t s0 = int64_t(t) * spt, s1 = std::min<int64_t>(s0 + spt, S.n_slices);
        const int64_t e0 = S.slice_ptr[s0], e1 = S.slice_ptr[s1];
        if (!one && e1 - e0 > 65535) return fail(DECBPM_ERR_UNSUPPORTED, "tile %d has %lld SELL entries", t, (long long)(e1 - e0));
        uniq.clear();
        for (int64_t e = e0; e < e1; ++e)
            if (S.col[e] < r0 || S.col[e] >= r1) uniq.push_back(S.col[e]);
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        if ((tile_rows + uniq.size()) * row_bytes > 65535) {   // window offsets must fit 16 bits: keep the row kernel
            T.ready = true;
            T.ok = false;
            return DECBPM_OK;
        }
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t q = S.col[e];
            const int64_t w = (q >= r0 && q < r1) ? q - r0
                                                  : tile_rows + (std::lower_bound(uniq.begin(), uniq.end(), q) - uniq.begin());
            lcol[e] = uint16_t(w * row_bytes);              // byte offset of the row in the window
        }
        int32_t *d = &desc[size_t(t) * 8];
        d[0] = int32_t(e0);
        d[1] = int32_t(e1 - e0);
        d[2] = int32_t(hovf.size());
        d[3] = int32_t(uniq.size());
        uint32_t es[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
        for (int64_t sl = s0; sl < s1 && !one; ++sl) {
            if (S.slice_w[sl] > 255) return fail(DECBPM_ERR_UNSUPPORTED, "slice %lld is wider than 255", (long long)sl);
            es[sl - s0] = uint32_t(S.slice_ptr[sl] - e0);
            w[sl - s0] = uint32_t(S.slice_w[sl]);
        }
        d[4] = int32_t(es[0] | es[1] << 16);
        d[5] = int32_t(es[2] | es[3] << 16);
        d[6] = int32_t(w[0] | w[1] << 8 | w[2] << 16 | w[3] << 24);
        for (size_t j = 0; j < uniq.size(); ++j) {
            if (j < size_t(held)) hfixed[size_t(t) * held + j] = uniq[j];
            else hovf.push_back(uniq[j]);
            const int32_t tq = uniq[j] / tile_rows;
            if (adj[t].empty() || adj[t].back() != tq) adj[t].push_back(tq);    // uniq is sorted
        }
        max_halo = std::max(max_halo, int(uniq.size()));
        max_entries = std::max(max_entries, int(e1 - e0));
    }
    // dependency lists of the dataflow march: the tile itself and every tile
    // adjacent to it, made symmetric (a tile whose rows another tile reads as
    // halo depends on that tile too), at most kDepInts - 1 entries
    std::vector<std::vector<int32_t>> dep(nt);
    for (int t = 0; t < nt; ++t) {
        dep[t].push_back(t);
        for (int32_t u : adj[t]) {
            dep[t].push_back(u);
            dep[u].push_back(t);
        }
    }
    std::vector<int32_t> tdeps(size_t(nt) * kDepInts, 0);
    bool flow_ok = true;
    for (int t = 0; t < nt && flow_ok; ++t) {
        std::vector<int32_t> &d = dep[t];
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
        if (int(d.size()) > kDepInts - 1) { flow_ok = false; break; }
        tdeps[size_t(t) * kDepInts] = int32_t(d.size());
        for (size_t j = 0; j < d.size(); ++j) tdeps[size_t(t) * kDepInts + 1 + j] = d[j];
    }
    if (flow_ok) TRY(M->mem.upload(&T.tdeps, tdeps));
    T.flow_ok = flow_ok;
    TRY(M->mem.upload(&T.lcol, lcol));
    TRY(M->mem.upload(&T.tdesc, desc));
    TRY(M->mem.upload(&T.halo_rows, hfixed));
    TRY(M->mem.upload(&T.halo_ovf, hovf));
    T.n_tiles = nt;
    T.max_halo = max_halo;
    T.max_entries = max_entries;
    T.ready = true;
    T.ok = true;
    return DECBPM_OK;
}

// Stage-pair maps of the 128-row tiles (see march_pair_kernel): H1 = the
// tile's neighbour rows outside it (sorted; the same order as the tile maps'
// halo, so the tile's own window offsets stay valid), H2 = the neighbour rows
// of H1 outside tile + H1 (sorted).  Per tile: the list [H1, H2] at a fixed
// place kPairHL t, a descriptor of kPairDesc int32 (see the kernel), and the
// SELL entries of the H1 rows in slices of 32 (each row's entries in the
// mesh's SELL order, window offsets into [tile, H1, H2] as row * 128 and the
// same FP32 x_pq, so a halo row's b_k is the one its owner computes).
// Meshes whose tiles exceed the capacities keep the single-stage kernels.
static int build_pair_maps(decbpm_mesh_t M) {
    if (M->pairs_ready) return DECBPM_OK;
    TRY(build_tiles(M));
    M->pairs_ready = true;
    M->pairs_ok = false;
    if (!M->t16.ok) return DECBPM_OK;
    const Sell &S = M->S;
    const Assembly &A = M->A;
    const int64_t n0 = A.n0;
    const int nt = int((n0 + kTileRows - 1) / kTileRows);
    constexpr int spt = kTileRows / kSlice;
    const double r = M->r();
    std::vector<int32_t> pdesc(size_t(nt) * kPairDesc, 0), hlist(size_t(nt) * kPairHL, 0);
    std::vector<uint16_t> lcol2;
    std::vector<float> x2;
    std::vector<int32_t> h1, h2;
    std::unordered_map<int32_t, int32_t> widx;
    int max_nh1 = 0, max_nh12 = 0, max_he = 0;
    for (int t = 0; t < nt; ++t) {
        const int64_t r0 = int64_t(t) * kTileRows, r1 = std::min<int64_t>(r0 + kTileRows, n0);
        const int64_t s0 = int64_t(t) * spt, s1 = std::min<int64_t>(s0 + spt, S.n_slices);
        const int64_t e0 = S.slice_ptr[s0], e1 = S.slice_ptr[s1];
        h1.clear();
        for (int64_t e = e0; e < e1; ++e)
            if (S.col[e] < r0 || S.col[e] >= r1) h1.push_back(S.col[e]);
        std::sort(h1.begin(), h1.end());
        h1.erase(std::unique(h1.begin(), h1.end()), h1.end());
        auto in_w1 = [&](int32_t q) { return (q >= r0 && q < r1) || std::binary_search(h1.begin(), h1.end(), q); };
        h2.clear();
        for (int32_t q : h1) {
            const int64_t sq = q >> 5, lq = q & 31;
            for (int j = 0; j < S.slice_w[sq]; ++j) {
                const int32_t c = S.col[S.slice_ptr[sq] + int64_t(j) * kSlice + lq];
                if (!in_w1(c)) h2.push_back(c);
            }
        }
        std::sort(h2.begin(), h2.end());
        h2.erase(std::unique(h2.begin(), h2.end()), h2.end());
        const int nh1 = int(h1.size()), nh2 = int(h2.size());
        if (nh1 > kPairH1 || nh1 + nh2 > kPairHL) return DECBPM_OK;     // capacity: keep single-stage kernels
        widx.clear();
        for (int i = 0; i < nh1; ++i) widx[h1[i]] = kTileRows + i;
        for (int i = 0; i < nh2; ++i) widx[h2[i]] = kTileRows + nh1 + i;
        auto wpos = [&](int32_t c) -> int32_t {
            if (c >= r0 && c < r1) return int32_t(c - r0);
            auto it = widx.find(c);
            return it == widx.end() ? -1 : it->second;
        };
        // H1 rows' SELL entries, slices of 32 halo rows
        const int he0 = int(lcol2.size());
        uint32_t hw[4] = {0, 0, 0, 0};
        const int nhs = (nh1 + kSlice - 1) / kSlice;
        for (int sl = 0; sl < nhs; ++sl) {
            int w = 0;
            for (int i = sl * kSlice; i < std::min(nh1, (sl + 1) * kSlice); ++i) w = std::max(w, int(S.slice_w[h1[i] >> 5]));
            if (w > 255) return DECBPM_OK;
            hw[sl] = uint32_t(w);
            const size_t base = lcol2.size();
            lcol2.resize(base + size_t(kSlice) * w, 0);
            x2.resize(base + size_t(kSlice) * w, 0.0f);
            for (int lane = 0; lane < kSlice; ++lane) {
                const int i = sl * kSlice + lane;
                const int32_t self = kTileRows + std::min(i, std::max(nh1 - 1, 0));
                for (int j = 0; j < w; ++j) {
                    const size_t o = base + size_t(j) * kSlice + lane;
                    lcol2[o] = uint16_t(self * 128);
                    x2[o] = 0.0f;
                    if (i >= nh1) continue;
                    const int32_t q = h1[i];
                    const int64_t sq = q >> 5, lq = q & 31;
                    if (j >= S.slice_w[sq]) continue;
                    const int64_t idx = S.slice_ptr[sq] + int64_t(j) * kSlice + lq;
                    const int32_t pos = wpos(S.col[idx]);
                    if (pos < 0) return fail(DECBPM_ERR_CUDA, "internal: halo neighbour outside the pair window");
                    lcol2[o] = uint16_t(pos * 128);
                    x2[o] = float(S.w[idx] / (r * A.m[A.perm[q]]));
                }
            }
        }
        const int hne = int(lcol2.size()) - he0;
        int32_t *d = &pdesc[size_t(t) * kPairDesc];
        d[0] = int32_t(e0);
        d[1] = int32_t(e1 - e0);
        d[2] = int32_t(nh1 | (nh2 << 16));
        d[3] = he0;
        uint32_t es[4] = {0, 0, 0, 0}, w[4] = {0, 0, 0, 0};
        for (int64_t sl = s0; sl < s1; ++sl) {
            es[sl - s0] = uint32_t(S.slice_ptr[sl] - e0);
            w[sl - s0] = uint32_t(S.slice_w[sl]);
        }
        d[4] = int32_t(es[0] | es[1] << 16);
        d[5] = int32_t(es[2] | es[3] << 16);
        d[6] = int32_t(w[0] | w[1] << 8 | w[2] << 16 | w[3] << 24);
        d[7] = int32_t(hw[0] | hw[1] << 8 | hw[2] << 16 | hw[3] << 24);
        d[8] = hne;
        for (int i = 0; i < nh1; ++i) hlist[size_t(t) * kPairHL + i] = h1[i];
        for (int i = 0; i < nh2; ++i) hlist[size_t(t) * kPairHL + nh1 + i] = h2[i];
        max_nh1 = std::max(max_nh1, nh1);
        max_nh12 = std::max(max_nh12, nh1 + nh2);
        max_he = std::max(max_he, hne);
    }
    if (lcol2.empty()) { lcol2.push_back(0); x2.push_back(0.0f); }
    TRY(M->mem.upload(&M->pdesc, pdesc));
    TRY(M->mem.upload(&M->hlist, hlist));
    TRY(M->mem.upload(&M->lcol2, lcol2));
    TRY(M->mem.upload(&M->x2, x2));
    M->max_nh1 = max_nh1;
    M->max_nh12 = max_nh12;
    M->max_hentries = max_he;
    M->pairs_ok = true;
    return DECBPM_OK;
}

static int mesh_upload(decbpm_mesh_t M) {
    const Assembly &A = M->A;
    const Sell &S = M->S;
    const int64_t n0 = A.n0;
    const double c = 0.5 * A.rho, r = 0.5 * A.rho;
    // X = (A - c)/r with A = *0^{-1} K and c = r:  X = A/r - I.  The fused
    // kernels store x_pq = w_pq / (r m_p) and evaluate (X g)_p = sum_q x_pq (g_p - g_q) - g_p;
    // the plain path stores X itself in CSR (X_pq = -x_pq, X_pp = (sum_q w_pq / m_p - c) / r).
    std::vector<double> xval(S.col.size()), xdiag(n0), wv(S.col.size()), cv(S.col.size());
    std::vector<double> m(n0), v(n0), chib(n0), sig(n0), cdiag(n0);
    for (int64_t sl = 0; sl < S.n_slices; ++sl)
        for (int j = 0; j < S.slice_w[sl]; ++j)
            for (int lane = 0; lane < kSlice; ++lane) {
                const int64_t idx = S.slice_ptr[sl] + int64_t(j) * kSlice + lane;
                const int64_t row = sl * kSlice + lane;
                const double mp = row < n0 ? A.m[A.perm[row]] : 1.0;
                xval[idx] = S.w[idx] / (r * mp);
                wv[idx] = S.w[idx];
                cv[idx] = S.c[idx];
            }
    for (int64_t i = 0; i < n0; ++i) {
        const int32_t o = A.perm[i];
        m[i] = A.m[o];
        xdiag[i] = (A.wsum[o] / A.m[o] - c) / r;
        v[i] = A.v[o];
        chib[i] = A.chib[o];
        sig[i] = A.sigma[o];
        cdiag[i] = A.c_diag[o];
    }
    DevAllocs &D = M->mem;
    // slice tables padded to a multiple of 16 entries (the single-field tiles
    // bulk-copy 16 slices' offsets and widths; padding: no entries)
    const size_t nsp = (S.slice_ptr.size() + 15) / 16 * 16;
    std::vector<int32_t> sp(S.slice_ptr), sw(S.slice_w);
    sp.resize(nsp, S.slice_ptr.back());
    sw.resize(nsp, 0);
    TRY(D.upload(&M->slice_ptr, sp));
    TRY(D.upload(&M->slice_w, sw));
    TRY(D.upload(&M->col, S.col));
    TRY(D.upload(&M->perm, A.perm));
    TRY(D.upload(&M->x32, cast<float>(xval)));
    TRY(D.upload(&M->v32, cast<float>(v)));
    TRY(D.upload(&M->chib32, cast<float>(chib)));
    TRY(D.upload(&M->sig32, cast<float>(sig)));
    TRY(D.upload(&M->coff32, cast<float>(cv)));
    TRY(D.upload(&M->cdiag32, cast<float>(cdiag)));
    TRY(D.upload(&M->x64, xval));
    TRY(D.upload(&M->v64, v));
    TRY(D.upload(&M->vbase64, v));
    TRY(D.upload(&M->chib64, chib));
    TRY(D.upload(&M->sig64, sig));
    TRY(D.upload(&M->coff64, cv));
    TRY(D.upload(&M->cdiag64, cdiag));
    TRY(D.upload(&M->w64, wv));
    TRY(D.upload(&M->m64, m));
    // CSR of X (diagonal included) in internal order for the plain path
    std::vector<int32_t> rp(n0 + 1, 0), cc;
    std::vector<double> vv;
    cc.reserve(A.col.size() + n0);
    vv.reserve(A.col.size() + n0);
    for (int64_t i = 0; i < n0; ++i) {
        const int32_t o = A.perm[i];
        std::vector<std::pair<int32_t, double>> row;
        row.push_back({int32_t(i), xdiag[i]});
        for (int64_t k = A.rowptr[o]; k < A.rowptr[o + 1]; ++k) row.push_back({A.iperm[A.col[k]], -A.w[k] / (r * A.m[o])});
        std::sort(row.begin(), row.end());
        for (auto &e : row) { cc.push_back(e.first); vv.push_back(e.second); }
        rp[i + 1] = int32_t(cc.size());
    }
    TRY(D.upload(&M->csr_ptr, rp));
    TRY(D.upload(&M->csr_col, cc));
    TRY(D.upload(&M->csr_val, vv));
    return DECBPM_OK;
}

// ============================================================== plans
// Fields per entry of a field group: the tile-staged kernels' row width.
constexpr int kGroupFields = 16;

struct decbpm_plan_s {
    // plan entries: meshes, fields per entry, and (below) one set of field
    // buffers each.  A complex64 plan with more than kGroupFields fields on
    // a mesh runs that mesh as consecutive entries of at most kGroupFields
    // fields (field groups) that share its operator, so every entry fits the
    // tile-staged kernels; user_* is the caller's view (its meshes and field
    // counts), ent_user / ent_f0 map an entry to the caller's mesh and to its
    // first field there.  Without groups entries and caller meshes coincide.
    std::vector<decbpm_mesh_t> meshes;
    std::vector<int32_t> B;
    std::vector<decbpm_mesh_t> user_meshes;
    std::vector<int32_t> user_B, ent_user, ent_f0;
    int bpad = 1, bpad_log2 = 0, precision = DECBPM_C64, fpt = 1;
    int device = 0, num_sms = 0;
    int block = 256, grid = 0;
    DevAllocs mem;
    std::vector<void *> psi, b0, b1, b2, user;   // user: device staging for the host-buffer entry points
    void *y_plain = nullptr;                     // SpMV result of the plain path
    char *adj_ws = nullptr;                      // adjoint workspace (checkpoints, segment states, cotangent)
    size_t adj_ws_bytes = 0;
    char *rk_ws = nullptr;                       // Dormand-Prince workspace (stages, states, norms)
    size_t rk_ws_bytes = 0;
    char *sol_ws = nullptr;                      // soliton iteration workspace
    size_t sol_ws_bytes = 0;
    void *views = nullptr, *coef = nullptr;
    int32_t *active = nullptr;
    int coef_cap = 0, active_cap = 0;
    unsigned long long *barrier = nullptr;
    int *status = nullptr;
    double *partial = nullptr, *diag_dev = nullptr, *diag_host = nullptr;   // diag_host pinned
    int diag_cap = 0;
    std::vector<int> diag_blocks;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // coefficient configuration
    double cfg_dz = 0, cfg_tol = -1;
    std::vector<int> order, M, item_begin, items;
    std::vector<double> theta0;                   // per mesh: phase left out of the step coefficients
    int S = 0, total_items = 0;
    // tile-staged march (complex64 with 9..16 fields)
    bool tile_mode = false;
    bool tile_one = false;                       // the single-field tiles (512 rows of one field)
    int tile_grid = 0, n_slots = 0, slot_bytes = 0, off_psi = 0, off_h = 0, off_lcol = 0, off_x = 0, off_hdr = 0;
    int slot_entries = 0;
    // launch configuration of the FUSED variant (defaults until decbpm_plan_autotune picks one)
    int max_per_sm = 1;                          // co-resident row-kernel CTAs per SM
    int tune_rows = 0;                           // 1: FUSED runs the row kernel even where tiles are possible
    int tune_slots = 0;                          // tile ring slots (0: all that fit)
    int forward_walk = 0;                        // 1: no reverse walk on odd stages
    bool tuned = false;
    std::vector<int> tile_begin;
    int32_t *active_tiles = nullptr;
    int active_tiles_cap = 0, total_tiles = 0;
    // stage-pair march (complex64, 16 fields): a fourth field buffer per mesh,
    // the slot layout, per-pass active tiles and per-stage coefficients
    bool pair_mode = false;
    int pair_slots = 0, pair_slot_bytes = 0, pair_grid = 0, n_passes = 0;
    int p_off_h = 0, p_off_psi = 0, p_off_lcol = 0, p_off_x = 0, p_off_lcol2 = 0, p_off_x2 = 0, p_off_hdr = 0;
    int p_slot_entries = 0, p_slot_hentries = 0, p_w2 = 0, p_w1 = 0;
    std::vector<void *> b3;
    int32_t *active_passes = nullptr;
    int active_passes_cap = 0;
    void *pcoef = nullptr;
    int pcoef_cap = 0;
    int tune_pair = -1;                          // 1: FUSED runs the stage-pair kernel; 0: not; -1: default
    // dataflow march (the tile-staged kernel without stage barriers): per-tile
    // counters, per-CTA tile lists of the current stage tables, the walk skip
    bool flow_mode = false;
    int flow_grid = 0;
    unsigned *tile_done = nullptr;
    int32_t *cta_tiles = nullptr, *cta_ptr = nullptr, *cta_cnt = nullptr, *active_meshes = nullptr;
    int cta_cnt_cap = 0, active_meshes_cap = 0;
    int tune_flow = 0;                           // 1: FUSED runs the dataflow kernel
    char *pml_st = nullptr;                      // stage table of the fused PML march
    size_t pml_st_bytes = 0;
    int tune_meta = 1;                           // row kernel, single-mesh plans: cache the item metadata
    // the last metadata-cache decision (row_meta_cache), so launches recorded
    // into a graph make no attribute or occupancy call
    const void *meta_fn = nullptr;
    int meta_grid = 0, meta_fpt = 0, meta_on = -1, meta_items = 0;
    size_t meta_dyn = 0;
    int flow_skip = kDefaultFlowSkip;
    int flow_ranges = 0;                         // dataflow kernel: 1 = contiguous ranges, 0 = chunk lists
    // graphs: key -> exec
    std::map<std::tuple<double, int64_t, int32_t, int32_t, double, int32_t>, cudaGraphExec_t> graphs;
    bool graphs_ok = true;
    ~decbpm_plan_s() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        if (diag_host) cudaFreeHost(diag_host);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (adj_ws) cudaFree(adj_ws);
        if (rk_ws) cudaFree(rk_ws);
        if (sol_ws) cudaFree(sol_ws);
        mem.release();
    }
};

// the tile maps a plan's tile-staged march uses
static const TileMaps &tile_maps(decbpm_plan_t P, decbpm_mesh_t m) { return P->tile_one ? m->t1 : m->t16; }

static int reject_pml(decbpm_mesh_t m);        // meshes with a PML run decbpm_propagate (one C128 field) and RK45 only
extern "C" {
static int single_plan(decbpm_mesh_t mesh, int64_t n_fields, int32_t precision, decbpm_plan_t *P,
                       bool field_groups = false);
}
static int reject_pml_plan(decbpm_plan_t P);

// Pinned host buffer for diagnostics of n_points points; graphs hold its
// address, so they are dropped when it moves.
static int ensure_diag_host(decbpm_plan_t P, int n_points) {
    if (n_points <= P->diag_cap && P->diag_host) return DECBPM_OK;
    for (auto &g : P->graphs) cudaGraphExecDestroy(g.second);
    P->graphs.clear();
    if (P->diag_host) cudaFreeHost(P->diag_host);
    P->diag_host = nullptr;
    P->diag_cap = 0;
    CK(cudaMallocHost(&P->diag_host, sizeof(double) * size_t(n_points) * P->meshes.size() * P->bpad * kDiagQ));
    P->diag_cap = n_points;
    return DECBPM_OK;
}

static size_t csize(int precision) { return precision == DECBPM_C64 ? 8 : 16; }

// The march kernel is instantiated per padded field count (1..64) and, for
// complex64 rows of four or more fields, per complex values per thread (4 or
// 2; the default is 4): fpt = 0 or the default picks the default instance.
static int default_fpt(int precision, int bpad) {
    return precision == DECBPM_C64 ? std::min(bpad, DECBPM_FPT4) : (bpad > 32 ? 2 : 1);
}
static bool fpt_allowed(int precision, int bpad, int fpt) {
    if (fpt == default_fpt(precision, bpad)) return true;
    return precision == DECBPM_C64 && bpad >= 4 && fpt == 2;
}
template <typename R> static const void *march_ptr_for(int bpad, int fpt = 0) {
    if constexpr (sizeof(R) == 4) {
        if (fpt == 2 && bpad >= 4) {
            switch (bpad) {
                case 4: return (const void *)march_kernel<float, 4, 2>;
                case 8: return (const void *)march_kernel<float, 8, 2>;
                case 16: return (const void *)march_kernel<float, 16, 2>;
                case 32: return (const void *)march_kernel<float, 32, 2>;
                default: return (const void *)march_kernel<float, 64, 2>;
            }
        }
    }
    switch (bpad) {
        case 1: return (const void *)march_kernel<R, 1>;
        case 2: return (const void *)march_kernel<R, 2>;
        case 4: return (const void *)march_kernel<R, 4>;
        case 8: return (const void *)march_kernel<R, 8>;
        case 16: return (const void *)march_kernel<R, 16>;
        case 32: return (const void *)march_kernel<R, 32>;
        default: return (const void *)march_kernel<R, 64>;
    }
}

static const void *march_kernel_ptr(int precision, int bpad, int fpt = 0) {
    return precision == DECBPM_C64 ? march_ptr_for<float>(bpad, fpt) : march_ptr_for<double>(bpad, fpt);
}

// Shared-memory metadata cache of the row kernel (see MetaCache): warp items
// per CTA and dynamic shared-memory bytes for a launch of `grid` CTAs, or
// {0, 0} for plans of several meshes (their stages' items differ), with the
// cache switched off, or when the CTAs would no longer all be co-resident.
constexpr size_t kMetaCacheMaxBytes = 96 * 1024;
static std::pair<int, size_t> row_meta_cache_eval(decbpm_plan_t P, const void *fn, int grid, int fpt) {
    if (P->meshes.size() != 1 || !P->tune_meta || grid < 1) return {0, 0};
    const size_t rs = P->precision == DECBPM_C64 ? sizeof(float) : sizeof(double);
    const int tpr = std::max(1, P->bpad / std::max(1, fpt));
    const int E = tpr >= 8 ? 1 : 8 / tpr;
    const int items = (P->total_items + grid - 1) / grid;
    size_t dyn = size_t(items) * E * 32 * (4 + rs) + size_t(items) * 4;
    dyn = (dyn + 15) / 16 * 16;
    if (items < 1 || dyn > kMetaCacheMaxBytes) return {0, 0};
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kMetaCacheMaxBytes)) != cudaSuccess)
        return {0, 0};
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, P->block, dyn) != cudaSuccess) return {0, 0};
    if (occ * P->num_sms < grid) return {0, 0};
    return {items, dyn};
}
static std::pair<int, size_t> row_meta_cache(decbpm_plan_t P, const void *fn, int grid, int fpt) {
    if (P->meta_fn != fn || P->meta_grid != grid || P->meta_fpt != fpt || P->meta_on != P->tune_meta) {
        const std::pair<int, size_t> r = row_meta_cache_eval(P, fn, grid, fpt);
        P->meta_fn = fn;
        P->meta_grid = grid;
        P->meta_fpt = fpt;
        P->meta_on = P->tune_meta;
        P->meta_items = r.first;
        P->meta_dyn = r.second;
    }
    return {P->meta_items, P->meta_dyn};
}

// Shared-memory ring of the tile-staged march: as many slots (3, else 2) of
// the largest tile window of the plan's meshes as fit next to the kernel's
// static shared memory.  Complex64 plans of 9..16 fields use 128-row tiles
// (march_tile_kernel), plans of one field per mesh 512-row tiles
// (march_tile1_kernel).  Plans it does not fit keep the row kernel.
static int setup_tiles(decbpm_plan_t P) {
    P->tile_mode = false;
    P->tile_one = false;
    if (P->precision != DECBPM_C64 || (P->bpad != 16 && P->bpad != 1)) return DECBPM_OK;
    const bool one = P->bpad == 1;
    int max_halo = 0, max_entries = 0;
    for (decbpm_mesh_t m : P->meshes) {
        TRY(build_tiles(m, one));
        const TileMaps &T = one ? m->t1 : m->t16;
        if (!T.ok) return DECBPM_OK;
        max_halo = std::max(max_halo, T.max_halo);
        max_entries = std::max(max_entries, T.max_entries);
    }
    auto up = [](int x) { return (x + 127) / 128 * 128; };
    const int row = one ? 8 : 16 * 8, rows = one ? kTile1Rows : kTileRows;
    P->off_psi = up((rows + max_halo) * row);
    P->off_h = P->off_psi + rows * row;
    P->off_lcol = P->off_h + rows * row;
    P->off_x = P->off_lcol + up(max_entries * 2);
    P->off_hdr = P->off_x + up(max_entries * 4);
    P->slot_entries = max_entries;
    P->slot_bytes = P->off_hdr + (one ? kTile1HdrBytes : 128);
    const void *fn = one ? (const void *)march_tile1_kernel : (const void *)march_tile_kernel;
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, fn));
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
    const int avail = optin - int(fa.sharedSizeBytes);
    P->n_slots = avail >= 3 * P->slot_bytes ? 3 : avail >= 2 * P->slot_bytes ? 2 : 0;
    if (P->n_slots == 0) return DECBPM_OK;
    const int dyn = P->n_slots * P->slot_bytes;
    // the attribute is per function, not per plan: allow the largest ring any plan may use
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, avail));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTileThreads, dyn));
    if (per_sm < 1) return DECBPM_OK;
    P->tile_grid = P->num_sms * per_sm;
    P->tile_mode = true;
    P->tile_one = one;
    // single-field plans run the row kernel until the autotuner picks the
    // tiles (faster on the 1M-vertex guide, slower on the L2-resident meshes
    // where the row kernel caches its metadata); no dataflow variant
    if (one) {
        P->tune_rows = 1;
        return DECBPM_OK;
    }
    // the dataflow kernel: same ring and static shared memory, one more warp
    P->flow_mode = false;
    bool deps_ok = true;
    int total = 0;
    for (decbpm_mesh_t m : P->meshes) {
        deps_ok = deps_ok && m->t16.flow_ok;
        total += m->t16.n_tiles;
    }
    if (!deps_ok) return DECBPM_OK;
    CK(cudaFuncGetAttributes(&fa, (const void *)march_flow_kernel));
    const int favail = optin - int(fa.sharedSizeBytes);
    if (favail < dyn) return DECBPM_OK;
    CK(cudaFuncSetAttribute((const void *)march_flow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, favail));
    int fper_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fper_sm, (const void *)march_flow_kernel, kFlowThreads, dyn));
    if (fper_sm < 1) return DECBPM_OK;
    P->flow_grid = P->num_sms * fper_sm;
    TRY(P->mem.alloc(&P->tile_done, size_t(total)));
    TRY(P->mem.alloc(&P->cta_ptr, size_t(P->flow_grid) + 1));
    TRY(P->mem.alloc(&P->cta_tiles, size_t(total)));
    P->flow_mode = true;
    return DECBPM_OK;
}

// Per-CTA tile lists of the dataflow march for the current plan order:
// every mesh's tiles are cut into grid contiguous chunks, in CTA order, whose
// sizes differ by at most one; the extra tiles of successive meshes go to
// successive CTAs (round robin), so every CTA's share of any prefix of the
// meshes differs from the others' by at most one tile.  A CTA's list holds
// its chunks of the meshes in plan order (meshes sorted by degree, so the
// meshes active in a stage are a prefix and a CTA's tiles of that stage a
// prefix of its list).
static int build_flow_lists(decbpm_plan_t P, const std::vector<int> &Ms) {
    const int n = int(P->meshes.size()), G = P->flow_grid;
    std::vector<std::vector<int32_t>> lists(G);
    std::vector<int32_t> cnt(size_t(G) * n, 0);
    int phi = 0;
    for (int j = 0; j < n; ++j) {
        const int i = P->order[j];
        const int T = P->meshes[i]->t16.n_tiles, q = T / G, r = T % G;
        int start = 0;
        for (int c = 0; c < G; ++c) {
            const bool extra = ((c - phi + G) % G) < r;
            const int sz = q + (extra ? 1 : 0);
            for (int u = 0; u < sz; ++u) lists[c].push_back(P->tile_begin[i] + start + u);
            start += sz;
            cnt[size_t(c) * n + j] = int32_t(lists[c].size());
        }
        phi = (phi + r) % G;
    }
    std::vector<int32_t> ptr(G + 1, 0), flat;
    flat.reserve(P->total_tiles);
    for (int c = 0; c < G; ++c) {
        ptr[c] = int32_t(flat.size());
        flat.insert(flat.end(), lists[c].begin(), lists[c].end());
    }
    ptr[G] = int32_t(flat.size());
    if (int(flat.size()) != P->total_tiles) return fail(DECBPM_ERR_CUDA, "dataflow tile lists are inconsistent");
    if (G * n > P->cta_cnt_cap) {
        TRY(P->mem.alloc(&P->cta_cnt, size_t(G) * n));
        P->cta_cnt_cap = G * n;
    }
    if (P->S > P->active_meshes_cap) {
        TRY(P->mem.alloc(&P->active_meshes, size_t(P->S)));
        P->active_meshes_cap = P->S;
    }
    std::vector<int32_t> am(P->S, 0);
    for (int s = 0; s < P->S; ++s)
        for (int j = 0; j < n; ++j)
            if (Ms[P->order[j]] > P->S - 1 - s) am[s] = j + 1;
    CK(cudaMemcpy(P->cta_tiles, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->cta_ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->cta_cnt, cnt.data(), sizeof(int32_t) * cnt.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->active_meshes, am.data(), sizeof(int32_t) * am.size(), cudaMemcpyHostToDevice));
    return DECBPM_OK;
}

// Shared-memory ring of the stage-pair march: two slots of the largest pair
// window of the plan's meshes (see march_pair_kernel).  Plans whose slots do
// not fit twice keep the single-stage kernels.
static int setup_pairs(decbpm_plan_t P) {
    P->pair_mode = false;
    if (!P->tile_mode || P->tile_one) return DECBPM_OK;
    int max_nh1 = 0, max_nh12 = 0, max_entries = 0, max_he = 0;
    for (decbpm_mesh_t m : P->meshes) {
        TRY(build_pair_maps(m));
        if (!m->pairs_ok) return DECBPM_OK;
        max_nh1 = std::max(max_nh1, m->max_nh1);
        max_nh12 = std::max(max_nh12, m->max_nh12);
        max_entries = std::max(max_entries, m->t16.max_entries);
        max_he = std::max(max_he, m->max_hentries);
    }
    auto up = [](int x) { return (x + 127) / 128 * 128; };
    const int row = 128;
    P->p_w2 = kTileRows + max_nh12;
    P->p_w1 = kTileRows + max_nh1;
    P->p_off_h = up(P->p_w2 * row);
    P->p_off_psi = P->p_off_h + up(P->p_w1 * row);
    P->p_off_lcol = P->p_off_psi + kTileRows * row;
    P->p_off_x = P->p_off_lcol + up(max_entries * 2);
    P->p_off_lcol2 = P->p_off_x + up(max_entries * 4);
    P->p_off_x2 = P->p_off_lcol2 + up(std::max(max_he, 1) * 2);
    P->p_off_hdr = P->p_off_x2 + up(std::max(max_he, 1) * 4);
    P->p_slot_entries = max_entries;
    P->p_slot_hentries = max_he;
    P->pair_slot_bytes = P->p_off_hdr + 128;
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, (const void *)march_pair_kernel));
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
    const int avail = optin - int(fa.sharedSizeBytes);
    P->pair_slots = avail >= 3 * P->pair_slot_bytes ? 3 : avail >= 2 * P->pair_slot_bytes ? 2 : 0;
    if (P->pair_slots == 0) return DECBPM_OK;
    CK(cudaFuncSetAttribute((const void *)march_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, avail));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)march_pair_kernel, kTileThreads,
                                                     P->pair_slots * P->pair_slot_bytes));
    if (per_sm < 1) return DECBPM_OK;
    P->pair_grid = P->num_sms * per_sm;
    const size_t cs = csize(P->precision);
    for (size_t i = 0; i < P->meshes.size(); ++i) {
        char *t;
        TRY(P->mem.alloc(&t, size_t(P->meshes[i]->A.n0) * P->bpad * cs));
        P->b3.push_back(t);
    }
    P->pair_mode = true;
    return DECBPM_OK;
}

static int plan_create_impl(const decbpm_mesh_t *meshes, int32_t n, const int32_t *fields, int32_t precision,
                            decbpm_plan_t *out, bool field_groups = false) {
    if (!out) return fail(DECBPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!meshes || !fields || n < 1 || n > kMaxMeshes)
        return fail(DECBPM_ERR_INVALID_ARG, "need 1..%d meshes with field counts", kMaxMeshes);
    if (precision != DECBPM_C64 && precision != DECBPM_C128) return fail(DECBPM_ERR_INVALID_ARG, "bad precision %d", precision);
    int maxB = 0;
    for (int i = 0; i < n; ++i) {
        if (!meshes[i]) return fail(DECBPM_ERR_INVALID_ARG, "mesh %d is NULL", i);
        if (fields[i] < 1 || fields[i] > kMaxFields)
            return fail(DECBPM_ERR_UNSUPPORTED, "fields per mesh must be in 1..%d (mesh %d has %d)", kMaxFields, i, fields[i]);
        maxB = std::max(maxB, int(fields[i]));
    }
    auto P = std::make_unique<decbpm_plan_s>();
    P->user_meshes.assign(meshes, meshes + n);
    P->user_B.assign(fields, fields + n);
    // entries: field groups of balanced sizes where they apply (and fit the
    // kernels' mesh table), else one entry per mesh
    auto make_entries = [&](bool split) {
        P->meshes.clear(); P->B.clear(); P->ent_user.clear(); P->ent_f0.clear();
        for (int i = 0; i < n; ++i) {
            const int g = split ? (fields[i] + kGroupFields - 1) / kGroupFields : 1;
            const int base = fields[i] / g, rem = fields[i] % g;
            for (int k = 0, f0 = 0; k < g; ++k) {
                const int b = base + (k < rem ? 1 : 0);
                P->meshes.push_back(meshes[i]);
                P->B.push_back(b);
                P->ent_user.push_back(i);
                P->ent_f0.push_back(f0);
                f0 += b;
            }
        }
    };
    make_entries(field_groups && precision == DECBPM_C64 && maxB > kGroupFields);
    if (int(P->meshes.size()) > kMaxMeshes) make_entries(false);
    maxB = *std::max_element(P->B.begin(), P->B.end());
    const int ne = int(P->meshes.size());
    P->precision = precision;
    P->bpad_log2 = ilog2(maxB);
    P->bpad = 1 << P->bpad_log2;
    // complex values per thread; must match Geo<R, BPAD, FPT>::FPT of the kernel launched
    P->fpt = default_fpt(precision, P->bpad);
    CK(cudaGetDevice(&P->device));
    CK(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));
    const size_t cs = csize(precision);
    P->user.assign(size_t(n), nullptr);
    for (int i = 0; i < ne; ++i) {
        // rows rounded up to a SELL slice: the single-field tiles bulk-copy an even row count
        const size_t elems = size_t((P->meshes[i]->A.n0 + kSlice - 1) / kSlice * kSlice) * P->bpad;
        void *a, *b, *c, *d;
        char *t;
        TRY(P->mem.alloc(&t, elems * cs)); a = t;
        TRY(P->mem.alloc(&t, elems * cs)); b = t;
        TRY(P->mem.alloc(&t, elems * cs)); c = t;
        TRY(P->mem.alloc(&t, elems * cs)); d = t;
        P->psi.push_back(a); P->b0.push_back(b); P->b1.push_back(c); P->b2.push_back(d);
        // deterministic diagnostic grid: depends on n0 and the SM count only
        const int rows_per_block = std::max(1, kDiagThreads >> P->bpad_log2);
        P->diag_blocks.push_back(int(std::min<int64_t>(2 * P->num_sms, (P->meshes[i]->A.n0 + rows_per_block - 1) / rows_per_block)));
    }
    char *t;
    TRY(P->mem.alloc(&t, precision == DECBPM_C64 ? sizeof(MeshView<float>) * ne : sizeof(MeshView<double>) * ne));
    P->views = t;
    TRY(P->mem.alloc(&P->barrier, 1));
    TRY(P->mem.alloc(&P->status, 1));
    CK(cudaMemset(P->status, 0, sizeof(int)));
    int maxdb = *std::max_element(P->diag_blocks.begin(), P->diag_blocks.end());
    TRY(P->mem.alloc(&P->partial, size_t(maxdb) * P->bpad * kDiagQ));
    TRY(P->mem.alloc(&P->diag_dev, size_t(ne) * P->bpad * kDiagQ));
    CK(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
    CK(cudaEventCreate(&P->ev0));
    CK(cudaEventCreate(&P->ev1));
    // occupancy-derived persistent grid: every CTA must be co-resident
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_kernel_ptr(precision, P->bpad), P->block, 0));
    if (per_sm < 1) return fail(DECBPM_ERR_CUDA, "march kernel cannot be resident with %d threads", P->block);
    P->max_per_sm = std::min(per_sm, 4);
    P->grid = P->num_sms * P->max_per_sm;
    TRY(setup_tiles(P.get()));
    TRY(setup_pairs(P.get()));
    *out = P.release();
    return DECBPM_OK;
}

// Chebyshev degrees and stage tables for one step length.
template <typename R>
static int plan_configure(decbpm_plan_t P, double dz, double tol) {
    if (P->cfg_dz == dz && P->cfg_tol == tol && !P->order.empty()) return DECBPM_OK;
    using C = typename CT<R>::c2;
    const int n = int(P->meshes.size());
    std::vector<Cheb> ch(n);
    for (int i = 0; i < n; ++i) TRY(cheb_coefficients(P->meshes[i]->A.p, P->meshes[i]->A.rho, dz, tol, ch[i]));
    P->order.resize(n);
    std::iota(P->order.begin(), P->order.end(), 0);
    std::stable_sort(P->order.begin(), P->order.end(), [&](int a, int b) { return ch[a].M > ch[b].M; });
    P->M.resize(n);
    P->theta0.resize(n);
    for (int i = 0; i < n; ++i) { P->M[i] = ch[i].M; P->theta0[i] = ch[i].theta0; }
    P->S = ch[P->order[0]].M;
    const int tpr_log2 = P->bpad_log2 - (P->fpt == 8 ? 3 : P->fpt == 4 ? 2 : P->fpt == 2 ? 1 : 0);
    const int rpw = 32 >> tpr_log2;
    P->item_begin.assign(n, 0);
    P->items.assign(n, 0);
    int acc = 0;
    for (int j = 0; j < n; ++j) {
        const int i = P->order[j];
        P->item_begin[i] = acc;
        P->items[i] = int((P->meshes[i]->A.n0 + rpw - 1) / rpw);
        acc += P->items[i];
    }
    P->total_items = acc;
    std::vector<int32_t> active_t(P->S, 0);
    if (P->tile_mode) {
        P->tile_begin.assign(n, 0);
        int tacc = 0;
        for (int j = 0; j < n; ++j) {
            const int i = P->order[j];
            P->tile_begin[i] = tacc;
            tacc += tile_maps(P, P->meshes[i]).n_tiles;
        }
        P->total_tiles = tacc;
        for (int s = 0; s < P->S; ++s)
            for (int j = 0; j < n; ++j)
                if (ch[P->order[j]].M > P->S - 1 - s) active_t[s] += tile_maps(P, P->meshes[P->order[j]]).n_tiles;
        if (P->S > P->active_tiles_cap) {
            TRY(P->mem.alloc(&P->active_tiles, P->S));
            P->active_tiles_cap = P->S;
        }
    }
    std::vector<int32_t> active(P->S);
    for (int s = 0; s < P->S; ++s) {
        const int k = P->S - 1 - s;
        int a = 0;
        for (int j = 0; j < n; ++j)
            if (ch[P->order[j]].M > k) a += P->items[P->order[j]];
        active[s] = a;
    }
    // stage tables (see StageCoef): fold b_M = a_M psi into the first two stages
    int total_coef = 0;
    for (int i = 0; i < n; ++i) total_coef += ch[i].M;
    if (total_coef > P->coef_cap) {
        char *t;
        TRY(P->mem.alloc(&t, sizeof(StageCoef<R>) * total_coef));
        P->coef = t;
        P->coef_cap = total_coef;
    }
    if (P->S > P->active_cap) {
        TRY(P->mem.alloc(&P->active, P->S));
        P->active_cap = P->S;
    }
    std::vector<StageCoef<R>> coef(total_coef);
    std::vector<MeshView<R>> views(n);
    int off = 0;
    auto mk = [](std::complex<double> z) { C c; c.x = R(z.real()); c.y = R(z.imag()); return c; };
    for (int j = 0; j < n; ++j) {
        const int i = P->order[j];
        const Cheb &cb = ch[i];
        const int Mi = cb.M;
        for (int k = 0; k < Mi; ++k) {
            StageCoef<R> s{};
            std::complex<double> alpha = cb.a[k], beta = (k == 0) ? 1.0 : 2.0;
            int flags = 0;
            if (k == Mi - 1) { flags |= kGisPsi; beta = 2.0 * cb.a[Mi]; }
            else if (k == Mi - 2) { alpha = cb.a[k] - cb.a[Mi]; }
            else flags |= kHasH;
            if (k == 0) flags |= kFinal;
            s.alpha = mk(alpha);
            s.beta = mk(beta);
            s.alpha_lo = mk(0.0);
            s.flags = flags;
            coef[off + k] = s;
        }
        // The kernel applies X to a constant field exactly (X 1 = -1), so the
        // lambda = 0 mode sees the stage recurrence at x = -1 with the stored
        // (rounded) coefficients.  Evaluate that recurrence in FP64 and put
        // the residual against the exact value f(lambda = 0) e^{-i theta0}
        // into alpha_lo: the smooth part of the field then carries no
        // systematic per-step phase or gain error from coefficient rounding.
        {
            auto up = [](C z) { return std::complex<double>(double(z.x), double(z.y)); };
            std::complex<double> bk1 = 0, bk2 = 0, Sv = 0;
            for (int k = Mi - 1; k >= 0; --k) {
                const StageCoef<R> &s = coef[off + k];
                const std::complex<double> g = (s.flags & kGisPsi) ? 1.0 : bk1;
                std::complex<double> o = up(s.alpha) - up(s.beta) * g;
                if (s.flags & kHasH) o -= bk2;
                if (s.flags & kFinal) Sv = o;
                bk2 = bk1;
                bk1 = o;
            }
            const std::complex<double> target = cb.f0;
            coef[off].alpha_lo = mk(target - Sv);
        }
        decbpm_mesh_t m = P->meshes[i];
        MeshView<R> &v = views[j];
        v.n0 = int32_t(m->A.n0);
        v.n_slices = int32_t(m->S.n_slices);
        v.M = Mi;
        v.item_begin = P->item_begin[i];
        v.slice_ptr = m->slice_ptr; v.slice_w = m->slice_w; v.col = m->col;
        if constexpr (sizeof(R) == 4) {
            v.xval = m->x32; v.v = m->v32; v.chib = m->chib32; v.sigma = m->sig32;
            v.coff = m->coff32; v.cdiag = m->cdiag32;
        } else {
            v.xval = m->x64; v.v = m->v64; v.chib = m->chib64; v.sigma = m->sig64;
            v.coff = m->coff64; v.cdiag = m->cdiag64;
        }
        v.psi = (C *)P->psi[i];
        v.b[0] = (C *)P->b0[i]; v.b[1] = (C *)P->b1[i]; v.b[2] = (C *)P->b2[i];
        v.coef = (const StageCoef<R> *)P->coef + off;
        if (P->tile_mode) {
            const TileMaps &T = tile_maps(P, m);
            v.lcol = T.lcol;
            v.tdesc = T.tdesc;
            v.halo_rows = T.halo_rows;
            v.halo_ovf = T.halo_ovf;
            v.tdeps = T.tdeps;
            v.tile_begin = P->tile_begin[i];
        }
        off += Mi;
    }
    if (P->flow_mode) {
        std::vector<int> Ms(n);
        for (int i = 0; i < n; ++i) Ms[i] = ch[i].M;
        TRY(build_flow_lists(P, Ms));
    }
    if (P->pair_mode) {
        // passes of a step: pairs (S-1, S-2), (S-3, S-4), ... down to stage 1, a
        // single pass for stage 1 when S - 1 is odd, the final stage 0; a mesh
        // takes part in a pass from its top stage M - 1 on (tiles: a prefix, the
        // meshes being sorted by degree)
        const int n_pairs = (P->S - 1) / 2;
        P->n_passes = n_pairs + ((P->S - 1) & 1) + 1;
        std::vector<int32_t> ap(P->n_passes, 0);
        for (int ps = 0; ps < P->n_passes; ++ps) {
            const int lowest = ps < n_pairs ? P->S - 2 - 2 * ps : (ps == n_pairs && ((P->S - 1) & 1)) ? 1 : 0;
            for (int j = 0; j < n; ++j)
                if (ch[P->order[j]].M > lowest) ap[ps] += P->meshes[P->order[j]]->t16.n_tiles;
        }
        if (P->n_passes > P->active_passes_cap) {
            TRY(P->mem.alloc(&P->active_passes, P->n_passes));
            P->active_passes_cap = P->n_passes;
        }
        CK(cudaMemcpy(P->active_passes, ap.data(), sizeof(int32_t) * P->n_passes, cudaMemcpyHostToDevice));
        if (sizeof(R) == 4) {
            if (total_coef > P->pcoef_cap) {
                char *t;
                TRY(P->mem.alloc(&t, sizeof(PairCoef) * total_coef));
                P->pcoef = t;
                P->pcoef_cap = total_coef;
            }
            std::vector<PairCoef> pc(total_coef);
            int o = 0;
            for (int j = 0; j < n; ++j) {
                const int Mi = ch[P->order[j]].M;
                for (int k = 0; k < Mi; ++k) {
                    const StageCoef<R> &sc = coef[o + k];
                    PairCoef c{};
                    c.alpha = make_float2(float(sc.alpha.x), float(sc.alpha.y));
                    c.beta = make_float2(float(sc.beta.x), float(sc.beta.y));
                    c.alpha_lo = make_float2(float(sc.alpha_lo.x), float(sc.alpha_lo.y));
                    c.flags = sc.flags;
                    if (k > 0) {
                        const StageCoef<R> &nx = coef[o + k - 1];
                        c.alpha_next = make_float2(float(nx.alpha.x), float(nx.alpha.y));
                        if (nx.flags & kHasH) c.flags |= kNextHasH;
                        if (nx.flags & kFinal) c.flags |= kNextFinal;
                    }
                    pc[o + k] = c;
                }
                views[j].pcoef = reinterpret_cast<const PairCoef *>(P->pcoef) + o;
                o += Mi;
            }
            CK(cudaMemcpy(P->pcoef, pc.data(), sizeof(PairCoef) * total_coef, cudaMemcpyHostToDevice));
        }
        for (int j = 0; j < n; ++j) {
            const int i = P->order[j];
            views[j].b3 = (C *)P->b3[i];
            views[j].pdesc = P->meshes[i]->pdesc;
            views[j].hlist = P->meshes[i]->hlist;
            views[j].lcol2 = P->meshes[i]->lcol2;
            views[j].x2 = P->meshes[i]->x2;
        }
    }
    if (P->tile_mode) CK(cudaMemcpy(P->active_tiles, active_t.data(), sizeof(int32_t) * P->S, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->coef, coef.data(), sizeof(StageCoef<R>) * total_coef, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->active, active.data(), sizeof(int32_t) * P->S, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->views, views.data(), sizeof(MeshView<R>) * n, cudaMemcpyHostToDevice));
    for (auto &g : P->graphs) cudaGraphExecDestroy(g.second);
    P->graphs.clear();
    P->cfg_dz = dz;
    P->cfg_tol = tol;
    return DECBPM_OK;
}

template <typename R>
static int launch_march(decbpm_plan_t P, cudaStream_t s, int n_steps, int kerr_mode, double dz, int variant) {
    MarchParams<R> mp{};
    mp.meshes = (const MeshView<R> *)P->views;
    mp.active_items = P->active;
    mp.n_meshes = int32_t(P->meshes.size());
    mp.S = P->S;
    mp.total_items = P->total_items;
    mp.n_steps = n_steps;
    mp.pre_half = 1;
    mp.post_half = 1;
    mp.kerr_mode = kerr_mode;
    mp.bpad_log2 = P->bpad_log2;
    mp.h = R(dz);
    mp.barrier = P->barrier;
    mp.status = P->status;
    mp.timeout_ns = kBarrierTimeoutNs;
    mp.forward_walk = P->forward_walk;
    CK(cudaMemsetAsync(P->barrier, 0, sizeof(unsigned long long), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P->grid);
    cfg.blockDim = dim3(P->block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&mp};
    const void *fn = march_ptr_for<R>(P->bpad, P->fpt);
    if constexpr (sizeof(R) == 4) {
        const bool pairs = P->pair_mode && (variant == DECBPM_VARIANT_PAIRS ||
                                            (variant == DECBPM_VARIANT_FUSED && !P->tune_rows && P->tune_pair == 1));
        if (pairs) {
            const int slots = (P->tune_pair == 1 && P->tune_slots > 0) ? std::min(P->tune_slots, P->pair_slots)
                                                                       : P->pair_slots;
            mp.active_tiles = P->active_passes;
            mp.n_passes = P->n_passes;
            mp.n_slots = slots;
            mp.slot_bytes = P->pair_slot_bytes;
            mp.off_psi = P->p_off_psi;
            mp.off_h = P->p_off_h;
            mp.off_lcol = P->p_off_lcol;
            mp.off_x = P->p_off_x;
            mp.off_lcol2 = P->p_off_lcol2;
            mp.off_x2 = P->p_off_x2;
            mp.off_hdr = P->p_off_hdr;
            mp.slot_entries = P->p_slot_entries;
            mp.slot_hentries = P->p_slot_hentries;
            mp.w2_rows = P->p_w2;
            mp.w1_rows = P->p_w1;
            cfg.gridDim = dim3(P->pair_grid);
            cfg.blockDim = dim3(kTileThreads);
            cfg.dynamicSmemBytes = size_t(slots) * P->pair_slot_bytes;
            void *pargs[] = {&mp};
            CK(cudaLaunchKernelExC(&cfg, (const void *)march_pair_kernel, pargs));
            return DECBPM_OK;
        }
        const bool flow = P->flow_mode && (variant == DECBPM_VARIANT_FLOW ||
                                           (variant == DECBPM_VARIANT_FUSED && !P->tune_rows && P->tune_pair != 1 &&
                                            P->tune_flow == 1));
        if (P->tile_mode && (variant == DECBPM_VARIANT_FUSED || variant == DECBPM_VARIANT_PAIRS || flow) &&
            !P->tune_rows) {
            const int slots = (P->tune_pair != 1 && P->tune_slots > 0) ? std::min(P->tune_slots, P->n_slots) : P->n_slots;
            mp.active_tiles = P->active_tiles;
            mp.n_slots = slots;
            mp.slot_bytes = P->slot_bytes;
            mp.off_psi = P->off_psi;
            mp.off_h = P->off_h;
            mp.off_lcol = P->off_lcol;
            mp.off_x = P->off_x;
            mp.off_hdr = P->off_hdr;
            mp.slot_entries = P->slot_entries;
            cfg.gridDim = dim3(P->tile_grid);
            cfg.blockDim = dim3(kTileThreads);
            cfg.dynamicSmemBytes = size_t(slots) * P->slot_bytes;
            fn = P->tile_one ? (const void *)march_tile1_kernel : (const void *)march_tile_kernel;
            if (flow) {
                mp.tile_done = P->tile_done;
                mp.cta_tiles = P->cta_tiles;
                mp.cta_ptr = P->cta_ptr;
                mp.cta_cnt = P->cta_cnt;
                mp.active_meshes = P->active_meshes;
                mp.flow_skip = P->flow_skip;
                mp.flow_ranges = P->flow_ranges;
                CK(cudaMemsetAsync(P->tile_done, 0, sizeof(unsigned) * size_t(P->total_tiles), s));
                cfg.gridDim = dim3(P->flow_grid);
                cfg.blockDim = dim3(kFlowThreads);
                fn = (const void *)march_flow_kernel;
            }
        }
    }
    if (fn == march_ptr_for<R>(P->bpad, P->fpt)) {
        const std::pair<int, size_t> mc = row_meta_cache(P, fn, int(cfg.gridDim.x), P->fpt);
        mp.meta_items = mc.first;
        cfg.dynamicSmemBytes = mc.second;
    }
    CK(cudaLaunchKernelExC(&cfg, fn, args));
    return DECBPM_OK;
}

template <typename R>
static int launch_diag(decbpm_plan_t P, cudaStream_t s, int kerr_mode, int point) {
    // writes diag_dev[mesh][f][q] and copies to diag_host[point][mesh][f][q]
    const int n = int(P->meshes.size());
    for (int i = 0; i < n; ++i) {
        decbpm_mesh_t m = P->meshes[i];
        diag_partial_kernel<R><<<P->diag_blocks[i], kDiagThreads, 0, s>>>(
            (const typename CT<R>::c2 *)P->psi[i], int32_t(m->A.n0), P->bpad_log2, P->B[i], m->slice_ptr, m->slice_w,
            m->col, m->w64, m->m64, m->v64, m->chib64, m->coff64, m->cdiag64, kerr_mode, P->partial);
        diag_final_kernel<<<P->B[i], kDiagThreads, 0, s>>>(P->partial, P->diag_blocks[i], P->bpad,
                                                            P->diag_dev + size_t(i) * P->bpad * kDiagQ);
    }
    CK(cudaGetLastError());
    const size_t per_point = size_t(n) * P->bpad * kDiagQ;
    CK(cudaMemcpyAsync(P->diag_host + per_point * point, P->diag_dev, per_point * sizeof(double), cudaMemcpyDeviceToHost, s));
    return DECBPM_OK;
}

// The device work of one propagate call: step blocks, diagnostics after each.
template <typename R>
static int enqueue_march(decbpm_plan_t P, cudaStream_t s, const decbpm_params *prm, int n_points) {
    const int64_t every = prm->diag_every > 0 ? prm->diag_every : std::max<int64_t>(prm->n_steps, 1);
    int64_t done = 0;
    int point = 0;
    bool first = true;
    while (done < prm->n_steps) {
        const int64_t nb = std::min<int64_t>(every, prm->n_steps - done);
        if (nb > 0x7fffffff) return fail(DECBPM_ERR_INVALID_ARG, "step block too long");
        if (first) CK(cudaEventRecordWithFlags(P->ev0, s, cudaEventRecordExternal));
        TRY(launch_march<R>(P, s, int(nb), prm->kerr_mode, prm->dz, prm->variant));
        if (done + nb >= prm->n_steps) CK(cudaEventRecordWithFlags(P->ev1, s, cudaEventRecordExternal));
        first = false;
        done += nb;
        TRY(launch_diag<R>(P, s, prm->kerr_mode, point++));
    }
    if (prm->n_steps == 0) {
        CK(cudaEventRecordWithFlags(P->ev0, s, cudaEventRecordExternal));
        CK(cudaEventRecordWithFlags(P->ev1, s, cudaEventRecordExternal));
        TRY(launch_diag<R>(P, s, prm->kerr_mode, point++));
    }
    (void)n_points;
    return DECBPM_OK;
}

static int n_diag_points(const decbpm_params *p) {
    if (p->n_steps == 0) return 1;
    if (p->diag_every <= 0) return 1;
    return int(p->n_steps / p->diag_every + (p->n_steps % p->diag_every ? 1 : 0));
}

static int check_params(const decbpm_params *p) {
    if (!p) return fail(DECBPM_ERR_INVALID_ARG, "params is NULL");
    if (!(p->dz > 0) || !std::isfinite(p->dz)) return fail(DECBPM_ERR_INVALID_ARG, "dz must be finite and > 0");
    if (p->n_steps < 0) return fail(DECBPM_ERR_INVALID_ARG, "n_steps < 0");
    if (p->precision != DECBPM_C64 && p->precision != DECBPM_C128) return fail(DECBPM_ERR_INVALID_ARG, "bad precision");
    if (p->kerr_mode != DECBPM_KERR_LUMPED && p->kerr_mode != DECBPM_KERR_ELEMENT) return fail(DECBPM_ERR_INVALID_ARG, "bad kerr_mode");
    if (p->diag_every < 0) return fail(DECBPM_ERR_INVALID_ARG, "diag_every < 0");
    if (p->variant != DECBPM_VARIANT_FUSED && p->variant != DECBPM_VARIANT_PLAIN && p->variant != DECBPM_VARIANT_ROWS &&
        p->variant != DECBPM_VARIANT_PAIRS && p->variant != DECBPM_VARIANT_FLOW)
        return fail(DECBPM_ERR_INVALID_ARG, "bad variant");
    if (!(p->cheb_tol >= 0)) return fail(DECBPM_ERR_INVALID_ARG, "cheb_tol < 0");
    return DECBPM_OK;
}

static double default_tol(const decbpm_params *p) {
    if (p->cheb_tol > 0) return p->cheb_tol;
    return p->precision == DECBPM_C64 ? 1e-9 : 1e-16;
}

static int finish_diag(decbpm_plan_t P, const decbpm_params *prm, int n_points, decbpm_diag *out) {
    const int n = int(P->meshes.size());
    bool finite = true;
    int rec = 0;
    const int64_t every = prm->diag_every > 0 ? prm->diag_every : std::max<int64_t>(prm->n_steps, 1);
    for (int pt = 0; pt < n_points; ++pt) {
        const int64_t steps_done = prm->n_steps == 0 ? 0 : std::min<int64_t>(prm->n_steps, (pt + 1) * every);
        for (int i = 0; i < n; ++i) {
            const std::vector<double> &p = P->meshes[i]->A.p;
            for (int f = 0; f < P->B[i]; ++f) {
                const double *q = P->diag_host + ((size_t(pt) * n + i) * P->bpad + f) * kDiagQ;
                decbpm_diag d;
                d.z = double(steps_done) * prm->dz;
                d.power = q[0];
                double lin = NAN;
                if (p.size() == 1) lin = p[0] * q[1];
                else if (p.size() == 2) lin = p[0] * q[1] - p[1] * q[2];
                d.hamiltonian = lin - q[3] - 0.5 * q[4];
                d.max_intensity = q[5];
                if (!std::isfinite(d.power) || !std::isfinite(d.max_intensity)) finite = false;
                if (out) out[rec] = d;
                ++rec;
            }
        }
    }
    if (!finite) return fail(DECBPM_ERR_NONFINITE, "field became non-finite (check dz, input amplitude and p_n)");
    return DECBPM_OK;
}

template <typename R>
static int plan_propagate_impl(decbpm_plan_t P, const decbpm_params *prm, void *const *psi_dev, cudaStream_t s,
                               decbpm_diag *diag_out) {
    using C = typename CT<R>::c2;
    const int n = int(P->meshes.size());
    TRY(plan_configure<R>(P, prm->dz, default_tol(prm)));
    const int n_points = n_diag_points(prm);
    TRY(ensure_diag_host(P, n_points));
    CK(cudaMemsetAsync(P->status, 0, sizeof(int), s));
    for (int i = 0; i < n; ++i) {
        const int64_t n0 = P->meshes[i]->A.n0;
        const int blocks = int(std::min<int64_t>(4 * P->num_sms, (n0 * P->bpad + 255) / 256));
        const int u = P->ent_user[i];
        permute_in_kernel<C><<<blocks, 256, 0, s>>>((const C *)psi_dev[u], (C *)P->psi[i], P->meshes[i]->perm,
                                                     int32_t(n0), P->B[i], P->bpad, P->user_B[u], P->ent_f0[i]);
    }
    CK(cudaGetLastError());
    // capture the march + diagnostics once per parameter set, replay afterwards
    // (the row kernel's metadata-cache decision is made here, not during capture)
    row_meta_cache(P, march_kernel_ptr(P->precision, P->bpad, P->fpt), P->grid, P->fpt);
    auto key = std::make_tuple(prm->dz, prm->n_steps, prm->diag_every, prm->kerr_mode, default_tol(prm), prm->variant);
    bool launched = false;
    if (P->graphs_ok) {
        auto it = P->graphs.find(key);
        if (it == P->graphs.end()) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            bool ok = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            int rc = DECBPM_OK;
            if (ok) rc = enqueue_march<R>(P, P->cap_stream, prm, n_points);
            cudaError_t ec = ok ? cudaStreamEndCapture(P->cap_stream, &g) : cudaErrorUnknown;
            if (ok && rc == DECBPM_OK && ec == cudaSuccess && g &&
                cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) {
                it = P->graphs.emplace(key, ge).first;
            } else {
                P->graphs_ok = false;   // capture unsupported here: launch directly from now on
                cudaGetLastError();
            }
            if (g) cudaGraphDestroy(g);
        }
        if (it != P->graphs.end()) {
            CK(cudaGraphLaunch(it->second, s));
            launched = true;
        }
    }
    if (!launched) TRY(enqueue_march<R>(P, s, prm, n_points));
    for (int i = 0; i < n; ++i) {
        const int64_t n0 = P->meshes[i]->A.n0;
        const int blocks = int(std::min<int64_t>(4 * P->num_sms, (n0 * P->B[i] + 255) / 256));
        const double ph = std::fmod(double(prm->n_steps) * P->theta0[i], 2.0 * M_PI);
        const int u = P->ent_user[i];
        permute_out_kernel<C><<<blocks, 256, 0, s>>>((const C *)P->psi[i], (C *)psi_dev[u], P->meshes[i]->perm,
                                                      int32_t(n0), P->B[i], P->bpad, std::cos(ph), std::sin(ph),
                                                      P->user_B[u], P->ent_f0[i]);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    int status = 0;
    CK(cudaMemcpy(&status, P->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status == DECBPM_ERR_TIMEOUT) return fail(DECBPM_ERR_TIMEOUT, "grid barrier timed out in the march kernel");
    if (status != 0) return fail(status, "device reported status %d", status);
    return finish_diag(P, prm, n_points, diag_out);
}

static int plan_propagate_dispatch(decbpm_plan_t P, const decbpm_params *prm, void *const *psi_dev, void *stream,
                                   decbpm_diag *diag_out) {
    TRY(check_params(prm));
    if (!P) return fail(DECBPM_ERR_INVALID_ARG, "plan is NULL");
    TRY(reject_pml_plan(P));
    if (!psi_dev) return fail(DECBPM_ERR_INVALID_ARG, "psi_dev is NULL");
    for (size_t i = 0; i < P->user_meshes.size(); ++i)
        if (!psi_dev[i]) return fail(DECBPM_ERR_INVALID_ARG, "psi_dev[%zu] is NULL", i);
    if (prm->precision != P->precision) return fail(DECBPM_ERR_INVALID_ARG, "params precision differs from the plan's");
    if (prm->variant == DECBPM_VARIANT_PLAIN) return fail(DECBPM_ERR_UNSUPPORTED, "plans run the fused variants only");
    if (P->precision == DECBPM_C64) return plan_propagate_impl<float>(P, prm, psi_dev, (cudaStream_t)stream, diag_out);
    return plan_propagate_impl<double>(P, prm, psi_dev, (cudaStream_t)stream, diag_out);
}

// ============================================================== plain FP64 path
struct PlainWork {
    double2 *psi = nullptr, *y = nullptr, *b[3] = {nullptr, nullptr, nullptr};
};

static int propagate_plain(decbpm_mesh_t m, const decbpm_params *prm, void *psi_dev, cudaStream_t s, decbpm_diag *diag_out) {
    if (prm->precision != DECBPM_C128) return fail(DECBPM_ERR_UNSUPPORTED, "the plain variant is FP64 (C128) only");
    const int n0 = int(m->A.n0);
    Cheb cb;
    TRY(cheb_coefficients(m->A.p, m->A.rho, prm->dz, default_tol(prm), cb));
    // one-field C128 plan for buffers, permutation and diagnostics
    decbpm_plan_t P = nullptr;
    auto key = std::make_pair(1, int(DECBPM_C128));
    auto it = m->plans.find(key);
    if (it == m->plans.end()) {
        int32_t one = 1;
        TRY(plan_create_impl(&m, 1, &one, DECBPM_C128, &P));
        m->plans[key] = P;
    } else P = it->second;
    TRY(plan_configure<double>(P, prm->dz, default_tol(prm)));
    double2 *psi = (double2 *)P->psi[0];
    double2 *b[3] = {(double2 *)P->b0[0], (double2 *)P->b1[0], (double2 *)P->b2[0]};
    if (!P->y_plain) {
        char *t;
        TRY(P->mem.alloc(&t, size_t(n0) * 16));
        P->y_plain = t;
    }
    double2 *y = (double2 *)P->y_plain;
    const int n_points = n_diag_points(prm);
    TRY(ensure_diag_host(P, n_points));
    const int T = 256, G = (n0 + T - 1) / T;
    permute_in_kernel<double2><<<std::min(G, 4 * P->num_sms), T, 0, s>>>((const double2 *)psi_dev, psi, m->perm, n0, 1, 1);
    const int64_t every = prm->diag_every > 0 ? prm->diag_every : std::max<int64_t>(prm->n_steps, 1);
    const int M = cb.M;
    int point = 0;
    CK(cudaEventRecord(P->ev0, s));
    for (int64_t step = 0; step < prm->n_steps; ++step) {
        const bool block_start = (step % every) == 0;
        const bool block_end = ((step + 1) % every) == 0 || step + 1 == prm->n_steps;
        if (block_start)
            plain_diag_flow_kernel<<<G, T, 0, s>>>(psi, m->v64, m->chib64, m->sig64, 0.5 * prm->dz, n0);
        for (int k = M - 1; k >= 0; --k) {
            std::complex<double> alpha = cb.a[k], beta = (k == 0) ? 1.0 : 2.0;
            int has_h = 1;
            const double2 *g = b[(k + 1) % 3];
            if (k == M - 1) { g = psi; beta = 2.0 * cb.a[M]; has_h = 0; }
            else if (k == M - 2) { alpha = cb.a[k] - cb.a[M]; has_h = 0; }
            plain_spmv_kernel<<<G, T, 0, s>>>(m->csr_ptr, m->csr_col, m->csr_val, g, y, n0);
            double2 *outp = (k == 0) ? psi : b[k % 3];
            plain_update_kernel<<<G, T, 0, s>>>(psi, y, b[(k + 2) % 3], outp, make_double2(alpha.real(), alpha.imag()),
                                                make_double2(beta.real(), beta.imag()), has_h, n0);
        }
        plain_diag_flow_kernel<<<G, T, 0, s>>>(psi, m->v64, m->chib64, m->sig64, block_end ? 0.5 * prm->dz : prm->dz, n0);
        if (block_end) {
            if (step + 1 == prm->n_steps) CK(cudaEventRecord(P->ev1, s));
            TRY(launch_diag<double>(P, s, DECBPM_KERR_LUMPED, point++));
        }
    }
    if (prm->n_steps == 0) {
        CK(cudaEventRecord(P->ev1, s));
        TRY(launch_diag<double>(P, s, DECBPM_KERR_LUMPED, point++));
    }
    const double ph = std::fmod(double(prm->n_steps) * cb.theta0, 2.0 * M_PI);
    permute_out_kernel<double2><<<std::min(G, 4 * P->num_sms), T, 0, s>>>(psi, (double2 *)psi_dev, m->perm, n0, 1, 1,
                                                                         std::cos(ph), std::sin(ph));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return finish_diag(P, prm, n_points, diag_out);
}


// ============================================================== adjoint (vector-Jacobian product)
// Reverse-mode derivative of psi_N = (D_{h/2} E_h D_{h/2})^N psi_0 (lumped Kerr):
// forward march with a checkpoint every C steps; backward segment by
// segment: recompute the segment's states one step at a time (each stored),
// then for every step, last first: adjoint of the trailing D_{h/2}, E_h^{-1}
// (the march kernel with -dz coefficients and the diagonal flow switched
// off: D_0 is the identity), adjoint of the leading D_{h/2}.
// With target_dev (decbpm_adjoint) the terminal cotangent is that of the
// overlap objective J_f = |<phi_f, psi_N,f>_{*0}|^2, formed on the device from
// the forward result (FP64 overlap, fixed-order reduction); J_out receives J_f.
template <typename R>
static int vjp_impl(decbpm_mesh_t mesh, decbpm_plan_t P, const decbpm_params *prm, const void *psi0_dev,
                    const void *gN_dev, void *psiN_dev, void *grad_psi0_dev, double *grad_v_dev, int64_t n_fields,
                    int32_t ck_every, cudaStream_t s, const void *target_dev = nullptr, double *J_out = nullptr) {
    using C = typename CT<R>::c2;
    const int64_t N = prm->n_steps;
    const int64_t n0 = mesh->A.n0;
    const int bpad = P->bpad;
    const double tol = default_tol(prm);
    TRY(plan_configure<R>(P, prm->dz, tol));
    Cheb cb_fwd, cb_bwd;
    TRY(cheb_coefficients(mesh->A.p, mesh->A.rho, prm->dz, tol, cb_fwd));
    TRY(cheb_coefficients(mesh->A.p, mesh->A.rho, -prm->dz, tol, cb_bwd));
    if (cb_bwd.M != cb_fwd.M) return fail(DECBPM_ERR_CUDA, "internal: backward degree differs");
    const int64_t Cs = ck_every > 0 ? ck_every : std::max<int64_t>(1, int64_t(std::ceil(std::sqrt(double(std::max<int64_t>(N, 1))))));
    const int64_t n_ck = N > 0 ? (N + Cs - 1) / Cs : 0;
    const size_t state = size_t(n0) * bpad * sizeof(C);
    const int M = cb_bwd.M;
    // workspace: G | grad_v (double n0) | backward view | backward stage table | checkpoints | segment states (Cs + 1)
    const size_t off_gv = (state + 255) & ~size_t(255);
    const size_t off_view = off_gv + ((sizeof(double) * n0 + 255) & ~size_t(255));
    const size_t off_coef = off_view + 256 * ((sizeof(MeshView<R>) + 255) / 256);
    const size_t off_ck = off_coef + 256 * ((sizeof(StageCoef<R>) * M + 255) / 256);
    const size_t off_seg = off_ck + state * size_t(n_ck);
    const int ovl_blocks = int(std::min<int64_t>(2 * P->num_sms, (n0 + std::max(1, kDiagThreads >> P->bpad_log2) - 1) /
                                                                    std::max(1, kDiagThreads >> P->bpad_log2)));
    const size_t off_ovl = off_seg + state * size_t(Cs + 1);          // overlap partials, then c[bpad][2]
    const size_t need = off_ovl + sizeof(double) * 2 * size_t(bpad) * (size_t(ovl_blocks) + 1);
    if (need > P->adj_ws_bytes) {
        if (P->adj_ws) cudaFree(P->adj_ws);
        P->adj_ws = nullptr;
        P->adj_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&P->adj_ws, need);
        if (e != cudaSuccess) return fail(DECBPM_ERR_OOM, "adjoint workspace of %zu bytes: %s", need, cudaGetErrorString(e));
        P->adj_ws_bytes = need;
    }
    char *ws = P->adj_ws;
    C *G = reinterpret_cast<C *>(ws);
    double *gv = reinterpret_cast<double *>(ws + off_gv);
    auto ck = [&](int64_t j) { return reinterpret_cast<C *>(ws + off_ck + state * size_t(j)); };
    auto seg = [&](int64_t j) { return reinterpret_cast<C *>(ws + off_seg + state * size_t(j)); };
    // backward view: the plan's mesh view with -dz coefficients, acting on G
    {
        std::vector<StageCoef<R>> coef(M);
        auto mk = [](std::complex<double> z) { C c; c.x = R(z.real()); c.y = R(z.imag()); return c; };
        for (int k = 0; k < M; ++k) {
            StageCoef<R> sc{};
            std::complex<double> alpha = cb_bwd.a[k], beta = (k == 0) ? 1.0 : 2.0;
            int flags = 0;
            if (k == M - 1) { flags |= kGisPsi; beta = 2.0 * cb_bwd.a[M]; }
            else if (k == M - 2) { alpha = cb_bwd.a[k] - cb_bwd.a[M]; }
            else flags |= kHasH;
            if (k == 0) flags |= kFinal;
            sc.alpha = mk(alpha); sc.beta = mk(beta); sc.alpha_lo = mk(0.0); sc.flags = flags;
            coef[k] = sc;
        }
        auto up = [](C z) { return std::complex<double>(double(z.x), double(z.y)); };
        std::complex<double> bk1 = 0, bk2 = 0, Sv = 0;
        for (int k = M - 1; k >= 0; --k) {
            const std::complex<double> g = (coef[k].flags & kGisPsi) ? 1.0 : bk1;
            std::complex<double> o = up(coef[k].alpha) - up(coef[k].beta) * g;
            if (coef[k].flags & kHasH) o -= bk2;
            if (coef[k].flags & kFinal) Sv = o;
            bk2 = bk1;
            bk1 = o;
        }
        coef[0].alpha_lo = mk(cb_bwd.f0 - Sv);
        MeshView<R> v{};
        CK(cudaMemcpy(&v, P->views, sizeof(MeshView<R>), cudaMemcpyDeviceToHost));
        v.psi = G;
        v.coef = reinterpret_cast<const StageCoef<R> *>(ws + off_coef);
        CK(cudaMemcpy(ws + off_coef, coef.data(), sizeof(StageCoef<R>) * M, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ws + off_view, &v, sizeof(v), cudaMemcpyHostToDevice));
    }
    const MeshView<R> *bwd_view = reinterpret_cast<const MeshView<R> *>(ws + off_view);
    auto march = [&](const MeshView<R> *views, int steps, R h, int pre) -> int {
        MarchParams<R> mp{};
        mp.meshes = views;
        mp.active_items = P->active;
        mp.n_meshes = 1;
        mp.S = P->S;
        mp.total_items = P->total_items;
        mp.n_steps = steps;
        mp.pre_half = pre;
        mp.post_half = 1;
        mp.kerr_mode = DECBPM_KERR_LUMPED;
        mp.bpad_log2 = P->bpad_log2;
        mp.h = h;
        mp.barrier = P->barrier;
        mp.status = P->status;
        mp.timeout_ns = kBarrierTimeoutNs;
        CK(cudaMemsetAsync(P->barrier, 0, sizeof(unsigned long long), s));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(P->grid);
        cfg.blockDim = dim3(P->block);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {&mp};
        const void *fn = march_ptr_for<R>(bpad, P->fpt);
        const std::pair<int, size_t> mc = row_meta_cache(P, fn, P->grid, P->fpt);
        mp.meta_items = mc.first;
        cfg.dynamicSmemBytes = mc.second;
        CK(cudaLaunchKernelExC(&cfg, fn, args));
        return DECBPM_OK;
    };
    const MeshView<R> *fwd_view = reinterpret_cast<const MeshView<R> *>(P->views);
    const R *vv = sizeof(R) == 4 ? (const R *)mesh->v32 : (const R *)mesh->v64;
    const R *cb = sizeof(R) == 4 ? (const R *)mesh->chib32 : (const R *)mesh->chib64;
    const R *sg = sizeof(R) == 4 ? (const R *)mesh->sig32 : (const R *)mesh->sig64;
    C *psi = (C *)P->psi[0];
    const int T = 256;
    const int Gv = int((n0 + T - 1) / T);
    const int Gs = int(std::min<int64_t>(4 * P->num_sms, (n0 * bpad + T - 1) / T));
    CK(cudaMemsetAsync(P->status, 0, sizeof(int), s));
    // forward with checkpoints
    permute_in_kernel<C><<<Gs, T, 0, s>>>((const C *)psi0_dev, psi, mesh->perm, int32_t(n0), int32_t(n_fields), bpad);
    for (int64_t j = 0; j < n_ck; ++j) {
        CK(cudaMemcpyAsync(ck(j), psi, state, cudaMemcpyDeviceToDevice, s));
        TRY(march(fwd_view, int(std::min<int64_t>(Cs, N - j * Cs)), R(prm->dz), 1));
    }
    const double phN = std::fmod(double(N) * cb_fwd.theta0, 2.0 * M_PI);
    if (psiN_dev)
        permute_out_kernel<C><<<Gs, T, 0, s>>>(psi, (C *)psiN_dev, mesh->perm, int32_t(n0), int32_t(n_fields), bpad,
                                               std::cos(phN), std::sin(phN));
    // terminal cotangent in the internal (phase-free, *0-weighted) frame
    double *ovl_part = reinterpret_cast<double *>(ws + off_ovl);
    double *ovl_c = ovl_part + 2 * size_t(bpad) * ovl_blocks;
    if (target_dev) {
        overlap_partial_kernel<C><<<ovl_blocks, kDiagThreads, 0, s>>>(psi, (const C *)target_dev, mesh->perm, mesh->m64,
                                                                      int32_t(n0), P->bpad_log2, int32_t(n_fields),
                                                                      ovl_part);
        overlap_final_kernel<<<int(n_fields), kDiagThreads, 0, s>>>(ovl_part, ovl_blocks, bpad, ovl_c);
        target_cotangent_kernel<C><<<Gs, T, 0, s>>>((const C *)target_dev, ovl_c, mesh->perm, G, int32_t(n0),
                                                    int32_t(n_fields), bpad);
    } else {
        cotangent_in_kernel<C><<<Gs, T, 0, s>>>((const C *)gN_dev, G, mesh->perm, mesh->m64, int32_t(n0),
                                                int32_t(n_fields), bpad, std::cos(phN), -std::sin(phN));
    }
    CK(cudaMemsetAsync(gv, 0, sizeof(double) * n0, s));
    const R hh = R(0.5 * prm->dz);
    for (int64_t j = n_ck - 1; j >= 0; --j) {
        const int64_t len = std::min<int64_t>(Cs, N - j * Cs);
        CK(cudaMemcpyAsync(psi, ck(j), state, cudaMemcpyDeviceToDevice, s));
        for (int64_t t = 0; t < len; ++t) {
            CK(cudaMemcpyAsync(seg(t), psi, state, cudaMemcpyDeviceToDevice, s));
            TRY(march(fwd_view, 1, R(prm->dz), 1));
        }
        CK(cudaMemcpyAsync(seg(len), psi, state, cudaMemcpyDeviceToDevice, s));
        for (int64_t t = len - 1; t >= 0; --t) {
            adj_diag_kernel<R><<<Gv, T, 0, s>>>(G, seg(t + 1), 1, int32_t(n0), int32_t(n_fields), bpad, hh, vv, cb, sg,
                                                mesh->m64, gv);
            TRY(march(bwd_view, 1, R(0), 0));
            adj_diag_kernel<R><<<Gv, T, 0, s>>>(G, seg(t), 0, int32_t(n0), int32_t(n_fields), bpad, hh, vv, cb, sg,
                                                mesh->m64, gv);
        }
    }
    if (grad_psi0_dev)
        gradient_out_kernel<C><<<Gs, T, 0, s>>>(G, (C *)grad_psi0_dev, mesh->perm, mesh->m64, int32_t(n0),
                                                int32_t(n_fields), bpad);
    if (grad_v_dev) scatter_real_kernel<<<Gv, T, 0, s>>>(gv, grad_v_dev, mesh->perm, int32_t(n0));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    int status = 0;
    CK(cudaMemcpy(&status, P->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status == DECBPM_ERR_TIMEOUT) return fail(DECBPM_ERR_TIMEOUT, "grid barrier timed out in the march kernel");
    if (status != 0) return fail(status, "device reported status %d", status);
    if (target_dev && J_out) {
        std::vector<double> c(2 * size_t(n_fields));
        CK(cudaMemcpy(c.data(), ovl_c, sizeof(double) * c.size(), cudaMemcpyDeviceToHost));
        for (int64_t f = 0; f < n_fields; ++f) {
            J_out[f] = c[2 * f] * c[2 * f] + c[2 * f + 1] * c[2 * f + 1];
            if (!std::isfinite(J_out[f])) return fail(DECBPM_ERR_NONFINITE, "overlap objective of field %lld is not finite",
                                                      (long long)f);
        }
    }
    return DECBPM_OK;
}


// ============================================================== the paper's integrator
// Adaptive Dormand-Prince 5(4) on the DEC ODE of Eq. 10 (FP64, one field):
// the stages, the error estimate and its RMS norm run on the device; the
// step controller (same rules as the oracle's dopri5) runs on the host and
// reads one double per attempted step.
static const double kDpA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double kDpB4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

static int rk45_impl(decbpm_mesh_t mesh, decbpm_plan_t P, double z_end, int kerr_mode, const decbpm_rk45_opts *o,
                     void *psi_dev, cudaStream_t s, decbpm_rk45_stats *stats) {
    const int n0 = int(mesh->A.n0);
    const std::vector<double> &pp = mesh->A.p;
    if (pp.size() > 2) return fail(DECBPM_ERR_UNSUPPORTED, "the RK45 path supports p_1 and p_2");
    const double p1 = pp[0], p2 = pp.size() > 1 ? pp[1] : 0.0;
    const double r = 0.5 * mesh->A.rho;
    const int T = kRkThreads, G = (n0 + T - 1) / T;
    const int NB = std::min(2 * P->num_sms, G);
    const size_t vec = size_t(n0) * sizeof(double2);
    const size_t need = 11 * vec + sizeof(double) * (NB + 1);
    if (need > P->rk_ws_bytes) {
        if (P->rk_ws) cudaFree(P->rk_ws);
        P->rk_ws = nullptr;
        P->rk_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&P->rk_ws, need);
        if (e != cudaSuccess) return fail(DECBPM_ERR_OOM, "RK45 workspace of %zu bytes: %s", need, cudaGetErrorString(e));
        P->rk_ws_bytes = need;
    }
    double2 *K[7], *y, *ys, *tmp, *tA;
    for (int j = 0; j < 7; ++j) K[j] = reinterpret_cast<double2 *>(P->rk_ws + j * vec);
    y = reinterpret_cast<double2 *>(P->rk_ws + 7 * vec);
    ys = reinterpret_cast<double2 *>(P->rk_ws + 8 * vec);
    tmp = reinterpret_cast<double2 *>(P->rk_ws + 9 * vec);
    tA = reinterpret_cast<double2 *>(P->rk_ws + 10 * vec);
    double *part = reinterpret_cast<double *>(P->rk_ws + 11 * vec);
    double *nrm = part + NB;
    MeshView<double> mv{};
    CK(cudaMemcpy(&mv, P->views, sizeof(mv), cudaMemcpyDeviceToHost));
    permute_in_kernel<double2><<<std::min(G, 4 * P->num_sms), T, 0, s>>>((const double2 *)psi_dev, y, mesh->perm, n0, 1, 1);
    int64_t n_rhs = 0;
    auto rhs = [&](const double2 *in, double2 *out) -> int {
        if (mesh->pml_on) {
            const PmlOps po{mv.slice_ptr, mv.slice_w, mv.col, mesh->pml_a, mesh->pml_v, mesh->pml_chib, mv.sigma, n0};
            if (pp.size() == 1) {
                rk_rhs_pml_kernel<<<G, T, 0, s>>>(po, in, out, nullptr, 0, p1, p2);
            } else {
                rk_rhs_pml_kernel<<<G, T, 0, s>>>(po, in, out, tA, 1, p1, p2);
                rk_rhs_pml_kernel<<<G, T, 0, s>>>(po, in, out, tA, 2, p1, p2);
            }
        } else if (pp.size() == 1) {
            rk_rhs_kernel<<<G, T, 0, s>>>(mv, in, out, nullptr, 0, r, p1, p2, kerr_mode);
        } else {
            rk_rhs_kernel<<<G, T, 0, s>>>(mv, in, out, tA, 1, r, p1, p2, kerr_mode);
            rk_rhs_kernel<<<G, T, 0, s>>>(mv, in, out, tA, 2, r, p1, p2, kerr_mode);
        }
        ++n_rhs;
        CK(cudaGetLastError());
        return DECBPM_OK;
    };
    auto combine = [&](double2 *out, const double2 *base, double h, const double *a, double2 *const *ks, int nk) {
        RkCombine c{};
        for (int j = 0; j < nk; ++j) { c.k[j] = ks[j]; c.a[j] = a[j]; }
        c.nk = nk;
        rk_combine_kernel<<<G, T, 0, s>>>(out, base, h, c, n0);
    };
    auto norm = [&](const double2 *u, const double2 *yy, const double2 *y2, double &out) -> int {
        rk_norm_partial_kernel<<<NB, T, 0, s>>>(u, yy, y2, o->atol, o->rtol, n0, part);
        rk_norm_final_kernel<<<1, T, 0, s>>>(part, NB, nrm);
        double v = 0;
        CK(cudaMemcpyAsync(&v, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        out = std::sqrt(v / (2.0 * n0));
        return DECBPM_OK;
    };
    TRY(rhs(y, K[0]));
    double h = o->h0;
    if (!(h > 0)) {
        double d0, d1, d2;
        TRY(norm(y, y, nullptr, d0));
        TRY(norm(K[0], y, nullptr, d1));
        const double h_try = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        const double one = 1.0;
        double2 *k0p[1] = {K[0]};
        combine(ys, y, h_try, &one, k0p, 1);
        TRY(rhs(ys, K[1]));
        const double a2[2] = {1.0, -1.0};
        double2 *kk[2] = {K[1], K[0]};
        combine(tmp, nullptr, 1.0, a2, kk, 2);
        TRY(norm(tmp, y, nullptr, d2));
        d2 /= h_try;
        const double h1 = std::max(d1, d2) <= 1e-15 ? std::max(1e-6, h_try * 1e-3) : std::pow(0.01 / std::max(d1, d2), 0.2);
        h = std::min(100 * h_try, h1);
    }
    double z = 0.0, h_last = 0.0;
    int64_t n_acc = 0, n_rej = 0;
    const int64_t max_steps = o->max_steps > 0 ? o->max_steps : (int64_t(1) << 40);
    double E_b[7];
    for (int j = 0; j < 7; ++j) E_b[j] = (j < 6 ? kDpA[6][j] : 0.0) - kDpB4[j];
    while (z < z_end && n_acc + n_rej < max_steps) {
        h = std::min(h, z_end - z);
        bool rejected = false;
        while (true) {
            for (int st = 1; st < 7; ++st) {
                combine(ys, y, h, kDpA[st], K, st);
                TRY(rhs(ys, K[st]));
            }
            combine(tmp, nullptr, h, E_b, K, 7);
            double E;
            TRY(norm(tmp, y, ys, E));
            if (!std::isfinite(E)) return fail(DECBPM_ERR_NONFINITE, "RK45 error estimate is not finite");
            if (E <= 1.0) {
                double factor = E == 0.0 ? 10.0 : std::min(10.0, 0.9 * std::pow(E, -0.2));
                if (rejected) factor = std::min(1.0, factor);
                z += h;
                std::swap(y, ys);
                std::swap(K[0], K[6]);
                ++n_acc;
                h_last = h;
                h *= factor;
                break;
            }
            ++n_rej;
            rejected = true;
            h *= std::max(0.2, 0.9 * std::pow(E, -0.2));
            if (h < 1e-300) return fail(DECBPM_ERR_NONFINITE, "RK45 step size underflow");
        }
    }
    permute_out_kernel<double2><<<std::min(G, 4 * P->num_sms), T, 0, s>>>(y, (double2 *)psi_dev, mesh->perm, n0, 1, 1,
                                                                         1.0, 0.0);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    if (stats) {
        stats->n_accepted = n_acc;
        stats->n_rejected = n_rej;
        stats->n_rhs = n_rhs;
        stats->h_last = h_last;
        stats->z = z;
    }
    return DECBPM_OK;
}


// ============================================================== discrete soliton
// Fundamental nonlinear mode of power P: y <- e^{-tau (H(y) - lo)} y, renormalised,
// with H(y) = p1 A + diag(d(y)) frozen per iteration.  A fixed point satisfies
// e^{-tau H(y)} y = c y, i.e. H(y) y = mu y: the self-consistent eigenmode,
// without splitting bias.  Spectrum of H within [min d, max d + p1 rho].
static int soliton_impl(decbpm_mesh_t mesh, decbpm_plan_t P, const decbpm_soliton_opts *o, void *psi_dev,
                        cudaStream_t s, decbpm_soliton_stats *st) {
    const int n0 = int(mesh->A.n0);
    if (mesh->A.p.size() != 1 || !(mesh->A.p[0] > 0)) return fail(DECBPM_ERR_UNSUPPORTED, "the soliton solver takes p_1 > 0 only");
    const double p1 = mesh->A.p[0], rA = 0.5 * mesh->A.rho, p1rA = p1 * rA;
    const int T = kRkThreads, G = (n0 + T - 1) / T;
    const int NB = std::min(2 * P->num_sms, G);
    const size_t vec = size_t(n0) * sizeof(double2);
    const size_t need = 5 * vec + 2 * size_t(n0) * sizeof(double) + sizeof(double) * (2 * NB + 2);
    if (need > P->sol_ws_bytes) {
        if (P->sol_ws) cudaFree(P->sol_ws);
        P->sol_ws = nullptr;
        P->sol_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&P->sol_ws, need);
        if (e != cudaSuccess) return fail(DECBPM_ERR_OOM, "soliton workspace of %zu bytes: %s", need, cudaGetErrorString(e));
        P->sol_ws_bytes = need;
    }
    double2 *y = reinterpret_cast<double2 *>(P->sol_ws);
    double2 *B[3] = {y + n0, y + 2 * size_t(n0), y + 3 * size_t(n0)};
    double2 *hy = y + 4 * size_t(n0);
    double *d = reinterpret_cast<double *>(P->sol_ws + 5 * vec);
    double *Imix = d + n0;
    double *part = Imix + n0;
    double *hy_I = reinterpret_cast<double *>(hy);          // |y|^2 for the residual, in hy's space before H y is formed
    double *res = part + 2 * NB;
    MeshView<double> mv{};
    CK(cudaMemcpy(&mv, P->views, sizeof(mv), cudaMemcpyDeviceToHost));
    auto reduce = [&](int mode, const double2 *a, const double2 *b, const double *r, double mu, double out[2]) -> int {
        sol_reduce_partial_kernel<<<NB, T, 0, s>>>(mode, a, b, r, mesh->m64, mu, n0, part);
        sol_reduce_final_kernel<<<1, T, 0, s>>>(mode, part, NB, res);
        CK(cudaMemcpyAsync(out, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return DECBPM_OK;
    };
    auto normalise = [&]() -> int {
        double q[2];
        TRY(reduce(0, y, nullptr, nullptr, 0.0, q));
        if (!(q[0] > 0) || !std::isfinite(q[0])) return fail(DECBPM_ERR_NONFINITE, "soliton iteration: field power is %g", q[0]);
        sol_scale_kernel<<<G, T, 0, s>>>(y, std::sqrt(o->power / q[0]), n0);
        return DECBPM_OK;
    };
    permute_in_kernel<double2><<<std::min(G, 4 * P->num_sms), T, 0, s>>>((const double2 *)psi_dev, y, mesh->perm, n0, 1, 1);
    CK(cudaGetLastError());
    TRY(normalise());
    double mu = 0, resid = 1e300;
    int64_t it = 0, terms = 0;
    std::vector<double> sk;
    for (it = 1; it <= o->max_iter; ++it) {
        sol_mix_kernel<<<G, T, 0, s>>>(y, Imix, o->mix, it == 1, n0);
        sol_potential_kernel<<<G, T, 0, s>>>(mv, Imix, o->kerr_mode, d);
        double mm[2];
        TRY(reduce(3, nullptr, nullptr, d, 0.0, mm));
        const double lo = mm[0], hi = mm[1] + p1 * mesh->A.rho;
        const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo), a = o->tau * r;
        // e^{-tau (lambda - lo)} = e^{-a (x + 1)} = s_0 + 2 sum_k (-1)^k s_k T_k(x),  s_k = e^{-a} I_k(a)
        bessel_i_scaled(a, 1e-17, sk);
        const int M = int(sk.size()) - 1;
        terms += M + 1;
        auto coef = [&](int k) { return k == 0 ? sk[0] : 2.0 * ((k & 1) ? -sk[k] : sk[k]); };
        double2 *out = nullptr;
        if (M == 0) {
            sol_stage_kernel<<<G, T, 0, s>>>(mv, y, nullptr, nullptr, B[0], d, p1rA, c, 1.0 / r, coef(0), 0.0);
            out = B[0];
        } else {
            // b_M = c_M y;  b_k = c_k y + 2 X b_{k+1} - b_{k+2};  S = c_0 y + X b_1 - b_2
            int i1 = 0, i2 = 1, i0 = 2;                      // b_{k+1}, b_{k+2}, b_k
            sol_stage_kernel<<<G, T, 0, s>>>(mv, y, nullptr, nullptr, B[i1], d, p1rA, c, 1.0 / r, coef(M), 0.0);
            bool have2 = false;
            for (int k = M - 1; k >= 0; --k) {
                const double beta = k == 0 ? 1.0 : 2.0;
                sol_stage_kernel<<<G, T, 0, s>>>(mv, y, B[i1], have2 ? B[i2] : nullptr, B[i0], d, p1rA, c, 1.0 / r,
                                                 coef(k), beta);
                const int t = i2; i2 = i1; i1 = i0; i0 = t;
                have2 = true;
            }
            out = B[i1];
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(y, out, vec, cudaMemcpyDeviceToDevice, s));
        TRY(normalise());
        // convergence: Rayleigh quotient and residual at the new field (unmixed intensity)
        sol_mix_kernel<<<G, T, 0, s>>>(y, hy_I, 1.0, 1, n0);
        sol_potential_kernel<<<G, T, 0, s>>>(mv, hy_I, o->kerr_mode, d);
        sol_apply_h_kernel<<<G, T, 0, s>>>(mv, y, d, p1rA, hy);
        double q0[2], q1[2], q2[2];
        TRY(reduce(0, y, nullptr, nullptr, 0.0, q0));
        TRY(reduce(1, y, hy, nullptr, 0.0, q1));
        mu = q1[0] / q0[0];
        TRY(reduce(2, y, hy, nullptr, mu, q2));
        resid = std::sqrt(q2[0] / q0[0]);
        if (!std::isfinite(resid)) return fail(DECBPM_ERR_NONFINITE, "soliton iteration diverged");
        if (resid < o->tol) break;
    }
    permute_out_kernel<double2><<<std::min(G, 4 * P->num_sms), T, 0, s>>>(y, (double2 *)psi_dev, mesh->perm, n0, 1, 1,
                                                                         1.0, 0.0);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    if (st) {
        st->mu = mu;
        st->residual = resid;
        st->iterations = std::min<int64_t>(it, o->max_iter);
        st->cheb_terms = terms;
    }
    return DECBPM_OK;
}


// ============================================================== autotuner
// Launch shapes of the FUSED march picked by timing: for complex64 plans that
// can run the tile-staged kernel, {tile kernel with 3 or 2 ring slots, row
// kernel with 1..max CTAs per SM} x {reverse walk on odd stages, forward
// only}; otherwise the row kernel's CTAs per SM x walk order; plans the
// stage-pair kernel can run also time it with 3 or 2 slots.  The single-stage
// candidates perform the same arithmetic per row (bitwise identical
// results); the stage-pair kernel stores a_k psi - b_{k+2} in place of b_{k+2}
// and so rounds differently (same FP32 accuracy against the oracle), so a plan
// that picks it differs from the others at the level of FP32 rounding.  Each candidate runs one untimed launch
// and then the best of two timed launches of `trial_steps` steps on the
// plan's internal buffers (zeroed first: their contents are scratch between
// calls).  The winner is cached for the process, keyed by the meshes'
// content fingerprints, the field counts, the precision, dz and kerr_mode.
struct TuneChoice {
    int rows = 0, per_sm = 0, slots = 0, forward = 0, pair = 0, fpt = 0;
    double ms = 0.0;
    int flow = 0, skip = 0, nometa = 0, ranges = 0;
};
static std::mutex g_tune_mutex;
static std::map<std::string, TuneChoice> g_tune_cache;

static uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}
static std::string tune_key(decbpm_plan_t P, double dz, int kerr_mode) {
    std::string k;
    char buf[96];
    for (size_t i = 0; i < P->meshes.size(); ++i) {
        const decbpm_mesh_t m = P->meshes[i];
        uint64_t h = 1469598103934665603ull;
        h = fnv(h, &m->A.n0, sizeof(m->A.n0));
        h = fnv(h, &m->A.rho, sizeof(m->A.rho));
        h = fnv(h, m->S.slice_w.data(), m->S.slice_w.size() * sizeof(int32_t));
        h = fnv(h, m->S.col.data(), m->S.col.size() * sizeof(int32_t));
        h = fnv(h, m->A.p.data(), m->A.p.size() * sizeof(double));
        std::snprintf(buf, sizeof(buf), "%016llx:%d;", (unsigned long long)h, P->B[i]);
        k += buf;
    }
    std::snprintf(buf, sizeof(buf), "p%d|dz%.17g|k%d", P->precision, dz, kerr_mode);
    return k + buf;
}

static void apply_choice(decbpm_plan_t P, const TuneChoice &c) {
    const int fpt = c.fpt > 0 ? c.fpt : default_fpt(P->precision, P->bpad);
    if (fpt != P->fpt) {
        P->fpt = fpt;
        P->cfg_dz = 0;           // rows per warp item changed: the stage tables are rebuilt on the next call
        P->cfg_tol = -1;
    }
    P->tune_rows = c.rows;
    P->tune_pair = c.pair;
    P->tune_flow = c.flow;
    P->tune_meta = c.nometa ? 0 : 1;
    P->flow_skip = c.skip > 0 ? c.skip : kDefaultFlowSkip;
    P->flow_ranges = c.ranges;
    P->tune_slots = c.slots;
    P->forward_walk = c.forward;
    P->grid = P->num_sms * c.per_sm;
    P->tuned = true;
    for (auto &g : P->graphs) cudaGraphExecDestroy(g.second);   // captured launches carry the old shape
    P->graphs.clear();
}

static decbpm_tune_result tune_result(const TuneChoice &c, int trial_steps, int n_cand, int from_cache) {
    decbpm_tune_result r{};
    r.variant = c.rows ? DECBPM_VARIANT_ROWS : c.pair ? DECBPM_VARIANT_PAIRS : c.flow ? DECBPM_VARIANT_FLOW
                                                                                     : DECBPM_VARIANT_FUSED;
    r.walk_skip = c.flow ? c.skip : 0;
    r.no_meta_cache = c.nometa;
    r.flow_ranges = c.flow ? c.ranges : 0;
    r.ctas_per_sm = c.rows ? c.per_sm : 1;
    r.tile_slots = c.slots;
    r.forward_walk = c.forward;
    r.ms_per_step = c.ms / trial_steps;
    r.candidates = n_cand;
    r.from_cache = from_cache;
    r.values_per_thread = c.fpt;
    return r;
}

template <typename R>
static int autotune_impl(decbpm_plan_t P, double dz, int kerr_mode, int trial_steps, cudaStream_t s,
                         decbpm_tune_result *out) {
    TRY(plan_configure<R>(P, dz, P->precision == DECBPM_C64 ? 1e-9 : 1e-16));
    const std::string key = tune_key(P, dz, kerr_mode);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply_choice(P, it->second);
            if (out) *out = tune_result(it->second, trial_steps, 0, 1);
            return DECBPM_OK;
        }
    }
    const size_t cs = csize(P->precision);
    for (size_t i = 0; i < P->meshes.size(); ++i) {
        const size_t bytes = size_t(P->meshes[i]->A.n0) * P->bpad * cs;
        CK(cudaMemsetAsync(P->psi[i], 0, bytes, s));
        CK(cudaMemsetAsync(P->b0[i], 0, bytes, s));
        CK(cudaMemsetAsync(P->b1[i], 0, bytes, s));
        CK(cudaMemsetAsync(P->b2[i], 0, bytes, s));
        if (P->pair_mode) CK(cudaMemsetAsync(P->b3[i], 0, bytes, s));
    }
    std::vector<TuneChoice> cand;
    const int fpt0 = default_fpt(P->precision, P->bpad);
    for (int fw = 0; fw <= 1; ++fw) {
        if (P->pair_mode)
            for (int sl = P->pair_slots; sl >= 2; --sl) cand.push_back({0, 1, sl, fw, 1, fpt0, 0.0, 0, 0});
        if (P->tile_mode)
            for (int sl = P->n_slots; sl >= 2; --sl) cand.push_back({0, P->max_per_sm, sl, fw, 0, fpt0, 0.0, 0, 0});
        if (P->flow_mode) {       // the skip only shapes reversed walks
            for (int skip : (fw == 0 ? std::vector<int>{4, 8, 16} : std::vector<int>{kDefaultFlowSkip}))
                cand.push_back({0, P->max_per_sm, P->n_slots, fw, 0, fpt0, 0.0, 1, skip});
            cand.push_back({0, P->max_per_sm, P->n_slots, fw, 0, fpt0, 0.0, 1, kDefaultFlowSkip, 0, 1});
        }
        std::vector<int> fpts = {fpt0};
        if (fpt0 == 4 && fpt_allowed(P->precision, P->bpad, 2)) fpts.push_back(2);
        for (int fpt : fpts) {
            int occ = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, march_kernel_ptr(P->precision, P->bpad, fpt), P->block, 0));
            for (int ps = 1; ps <= std::min(occ, 4); ++ps) cand.push_back({1, ps, 0, fw, 0, fpt, 0.0, 0, 0});
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    TuneChoice best{};
    best.ms = 1e300;
    int rc = DECBPM_OK;
    for (TuneChoice &c : cand) {
        apply_choice(P, c);
        rc = plan_configure<R>(P, dz, P->precision == DECBPM_C64 ? 1e-9 : 1e-16);
        if (rc != DECBPM_OK) break;
        if (cudaMemsetAsync(P->status, 0, sizeof(int), s) != cudaSuccess) { rc = fail(DECBPM_ERR_CUDA, "memset failed"); break; }
        double t_best = 1e300;
        for (int rep = 0; rep < 3 && rc == DECBPM_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) { rc = fail(DECBPM_ERR_CUDA, "event record failed"); break; }
            rc = launch_march<R>(P, s, trial_steps, kerr_mode, dz, DECBPM_VARIANT_FUSED);
            if (rc != DECBPM_OK) break;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = fail(DECBPM_ERR_CUDA, "autotune trial failed"); break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) t_best = std::min(t_best, double(ms));   // the first launch is untimed
        }
        if (rc != DECBPM_OK) break;
        int status = 0;
        if (cudaMemcpy(&status, P->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = fail(DECBPM_ERR_CUDA, "status read failed");
            break;
        }
        if (status != 0) { rc = fail(status, "device reported status %d during autotuning", status); break; }
        c.ms = t_best;
        if (t_best < best.ms) best = c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != DECBPM_OK) return rc;
    apply_choice(P, best);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    if (out) *out = tune_result(best, trial_steps, int(cand.size()), 0);
    return DECBPM_OK;
}


// ============================================================== PML
// Radial exterior complex scaling of the Hodge stars about (x0, y0): beyond
// r_inner the radius continues into the complex plane, r~ = r + i int sigma,
// s = 1 + i sigma(r), sigma = sigma_max ((r - r_inner)/(r_outer - r_inner))^order.
// Per triangle (at its centroid) the Whitney inner product of *1 gets the
// tensor Lambda = (r~/(s r)) e_r e_r^T + (s r/r~) e_t e_t^T and *0 the factor
// J = s r~ / r; K~ = d0^T *1~ d0 is the P1 stiffness with Lambda (complex
// symmetric, zero row sums); v and chib keep their lumped definitions with
// the stretched *0.  The RK45 integrator uses A~ = *0~^{-1} K~ in difference
// form: (A~ g)_p = sum_q a_pq (g_p - g_q), a_pq = -K~_pq / m~_p.
static int reject_pml(decbpm_mesh_t m) {
    if (m && m->pml_on)
        return fail(DECBPM_ERR_UNSUPPORTED,
                    "this mesh has a PML: it runs with decbpm_propagate (one complex128 field, lumped Kerr, p_1) "
                    "and decbpm_rk45 only");
    return DECBPM_OK;
}
static int reject_pml_plan(decbpm_plan_t P) {
    if (P)
        for (decbpm_mesh_t m : P->meshes) TRY(reject_pml(m));
    return DECBPM_OK;
}

static int set_pml_impl(decbpm_mesh_t M, const decbpm_pml *o) {
    using cd = std::complex<double>;
    const Assembly &A = M->A;
    const Sell &S = M->S;
    if (A.dim != 2) return fail(DECBPM_ERR_UNSUPPORTED, "the PML is radial: 2D meshes only");
    if (!(o->r_outer > o->r_inner) || !(o->r_inner >= 0) || !(o->sigma_max >= 0) || o->order < 0 || o->order > 8 ||
        !std::isfinite(o->x0 + o->y0 + o->r_inner + o->r_outer + o->sigma_max))
        return fail(DECBPM_ERR_INVALID_ARG, "PML needs 0 <= r_inner < r_outer, sigma_max >= 0, order in 0..8");
    const int64_t n0 = A.n0, nc = int64_t(M->g_cells.size()) / 3;
    const double *X = M->g_coords.data();
    const int32_t *C = M->g_cells.data();
    std::vector<cd> mt(n0, 0.0), nv(n0, 0.0), nchi(n0, 0.0);
    std::unordered_map<uint64_t, cd> K;
    K.reserve(size_t(nc) * 3);
    auto key = [&](int32_t a, int32_t b) { return uint64_t(std::min(a, b)) * uint64_t(n0) + uint64_t(std::max(a, b)); };
    for (int64_t t = 0; t < nc; ++t) {
        const int32_t v[3] = {C[3 * t], C[3 * t + 1], C[3 * t + 2]};
        const double px[3] = {X[2 * v[0]], X[2 * v[1]], X[2 * v[2]]}, py[3] = {X[2 * v[0] + 1], X[2 * v[1] + 1], X[2 * v[2] + 1]};
        const double a2 = (px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]);
        const double area = 0.5 * std::fabs(a2);
        double g[3][2];
        for (int i = 0; i < 3; ++i) {             // grad lambda_i = perp(opposite edge) / (2 |t|), signed
            const int j = (i + 1) % 3, k = (i + 2) % 3;
            g[i][0] = (py[j] - py[k]) / a2;
            g[i][1] = (px[k] - px[j]) / a2;
        }
        const double cx = (px[0] + px[1] + px[2]) / 3.0 - o->x0, cy = (py[0] + py[1] + py[2]) / 3.0 - o->y0;
        const double r = std::hypot(cx, cy);
        const double u = std::max(0.0, (r - o->r_inner) / (o->r_outer - o->r_inner));
        const double sig = o->order > 0 ? o->sigma_max * std::pow(u, o->order) : (r > o->r_inner ? o->sigma_max : 0.0);
        const cd sc(1.0, sig);
        const cd rt(r, o->sigma_max * (o->r_outer - o->r_inner) * std::pow(u, o->order + 1) / (o->order + 1));
        cd L[2][2], J;
        if (r > 0) {
            const double er[2] = {cx / r, cy / r}, et[2] = {-cy / r, cx / r};
            const cd ar = rt / (sc * r), at = sc * r / rt;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) L[a][b] = ar * er[a] * er[b] + at * et[a] * et[b];
            J = sc * rt / r;
        } else {
            L[0][0] = L[1][1] = 1.0;
            L[0][1] = L[1][0] = 0.0;
            J = 1.0;
        }
        for (int i = 0; i < 3; ++i) {
            mt[v[i]] += J * area / 3.0;
            nv[v[i]] += J * area / 3.0 * M->g_V[t];
            nchi[v[i]] += J * area / 3.0 * M->g_chi[t];
            for (int j = i + 1; j < 3; ++j) {
                cd kij = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) kij += g[i][a] * L[a][b] * g[j][b];
                K[key(v[i], v[j])] += area * kij;
            }
        }
    }
    std::vector<double2> a_sell(S.col.size()), vv(n0), cc(n0);
    for (int64_t sl = 0; sl < S.n_slices; ++sl)
        for (int j = 0; j < S.slice_w[sl]; ++j)
            for (int lane = 0; lane < kSlice; ++lane) {
                const int64_t idx = S.slice_ptr[sl] + int64_t(j) * kSlice + lane, row = sl * kSlice + lane;
                cd a = 0.0;
                if (row < n0 && j < S.degree[row]) {
                    const int32_t o1 = A.perm[row], o2 = A.perm[S.col[idx]];
                    auto it = K.find(key(o1, o2));
                    if (it == K.end()) return fail(DECBPM_ERR_BAD_MESH, "PML assembly: edge %d-%d not found", o1, o2);
                    a = -it->second / mt[o1];
                }
                a_sell[idx] = make_double2(a.real(), a.imag());
            }
    for (int64_t i = 0; i < n0; ++i) {
        const int32_t oi = A.perm[i];
        const cd v = nv[oi] / mt[oi], c = nchi[oi] / mt[oi];
        vv[i] = make_double2(v.real(), v.imag());
        cc[i] = make_double2(c.real(), c.imag());
    }
    // Gershgorin discs of A~ in internal order: centre sum_q a_pq, radius sum_q |a_pq|
    double re_lo = 1e300, re_hi = -1e300, im_lo = 1e300, im_hi = -1e300;
    for (int64_t row = 0; row < n0; ++row) {
        const int64_t sl = row / kSlice, lane = row % kSlice;
        cd z = 0.0;
        double rad = 0.0;
        for (int j = 0; j < S.slice_w[sl]; ++j) {
            const double2 a = a_sell[S.slice_ptr[sl] + int64_t(j) * kSlice + lane];
            z += cd(a.x, a.y);
            rad += std::hypot(a.x, a.y);
        }
        re_lo = std::min(re_lo, z.real() - rad);
        re_hi = std::max(re_hi, z.real() + rad);
        im_lo = std::min(im_lo, z.imag() - rad);
        im_hi = std::max(im_hi, z.imag() + rad);
    }
    M->pml_re_lo = re_lo; M->pml_re_hi = re_hi; M->pml_im_lo = im_lo; M->pml_im_hi = im_hi;
    const double rr = 0.5 * (re_hi - re_lo);
    const double rinv = rr > 0 ? 1.0 / rr : 0.0;       // an empty box is refused by the split-step
    std::vector<double2> x64(a_sell.size());
    std::vector<float2> x32(a_sell.size()), v32(n0), c32(n0);
    for (size_t i = 0; i < a_sell.size(); ++i) {
        x64[i] = make_double2(a_sell[i].x * rinv, a_sell[i].y * rinv);
        x32[i] = make_float2(float(x64[i].x), float(x64[i].y));
    }
    for (int64_t i = 0; i < n0; ++i) {
        v32[i] = make_float2(float(vv[i].x), float(vv[i].y));
        c32[i] = make_float2(float(cc[i].x), float(cc[i].y));
    }
    if (!M->pml_a) {
        TRY(M->mem.alloc(&M->pml_a, a_sell.size()));
        TRY(M->mem.alloc(&M->pml_v, size_t(n0)));
        TRY(M->mem.alloc(&M->pml_chib, size_t(n0)));
        TRY(M->mem.alloc(&M->pml_x64, a_sell.size()));
        TRY(M->mem.alloc(&M->pml_x32, a_sell.size()));
        TRY(M->mem.alloc(&M->pml_v32, size_t(n0)));
        TRY(M->mem.alloc(&M->pml_chib32, size_t(n0)));
    }
    CK(cudaMemcpy(M->pml_a, a_sell.data(), sizeof(double2) * a_sell.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(M->pml_v, vv.data(), sizeof(double2) * n0, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(M->pml_chib, cc.data(), sizeof(double2) * n0, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(M->pml_x64, x64.data(), sizeof(double2) * x64.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(M->pml_x32, x32.data(), sizeof(float2) * x32.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(M->pml_v32, v32.data(), sizeof(float2) * n0, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(M->pml_chib32, c32.data(), sizeof(float2) * n0, cudaMemcpyHostToDevice));
    M->pml_on = true;
    return DECBPM_OK;
}

// ============================================================== split-step with a PML
// The Strang march on the complex-stretched operators (one mesh, any number
// of fields, complex64 or complex128, lumped Kerr, p_1 only).
// E_h = exp(-i h p1 A~) is the Chebyshev series of exp(-i a x), a = h p1 r,
// in x = (lambda - c) / r over the real extent [c - r, c + r] of the
// Gershgorin region of A~; the series of this entire function converges on
// the complex spectrum too, and its degree is the smallest M whose tail
// sum_{k>M} 2 |J_k(a)| rho_e^k is below tol, rho_e the largest
// Bernstein-ellipse parameter of the region's box (so the truncation holds on
// every eigenvalue the box contains).  The stages run as one persistent
// launch per step block (pml_march_kernel) where one thread per (vertex,
// field) element fits the grid, else one launch per Chebyshev term and per
// diagonal flow.
// The Chebyshev series of E_h on the stretched operator's spectral box:
// centre c and half width r of the box's real extent, degree M, the
// coefficients coef_k of exp(-i a x) (a = h p1 r) and the phase theta0 the
// series leaves out: exp(-i h p1 lambda) = e^{i theta0} sum_k coef_k T_k(x).
struct PmlSeries {
    double c = 0, r = 0, theta0 = 0;
    int M = 0;
    std::vector<std::complex<double>> coef;
};
static int pml_series(decbpm_mesh_t m, double dz, double tol, PmlSeries &out) {
    using cd = std::complex<double>;
    if (!m->pml_on) return fail(DECBPM_ERR_INVALID_ARG, "the mesh has no PML");
    if (m->A.p.size() != 1) return fail(DECBPM_ERR_UNSUPPORTED, "with a PML the split-step takes p_1 only");
    const double p1 = m->A.p[0];
    const double lo = m->pml_re_lo, hi = m->pml_re_hi;
    const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
    if (!(r > 0)) return fail(DECBPM_ERR_BAD_MESH, "PML operator has an empty spectral box");
    // largest Bernstein-ellipse parameter over the boundary of the box
    double rho_e = 1.0;
    const double ylo = m->pml_im_lo / r, yhi = m->pml_im_hi / r;
    auto bern = [](cd x) {
        const cd w = x + std::sqrt(x * x - 1.0);
        return std::max(std::abs(w), 1.0 / std::abs(w));
    };
    for (int i = 0; i <= 400; ++i) {
        const double t = -1.0 + 2.0 * i / 400.0, u = ylo + (yhi - ylo) * i / 400.0;
        rho_e = std::max({rho_e, bern(cd(t, ylo)), bern(cd(t, yhi)), bern(cd(-1.0, u)), bern(cd(1.0, u))});
    }
    rho_e *= 1.01;
    const double a = dz * p1 * r;
    int kmax = int(std::fabs(a) * rho_e + 60 + 12 * std::cbrt(std::fabs(a) + 1.0));
    int M = 0;
    std::vector<double> J;
    for (;; kmax *= 2) {
        if (kmax > 200000) return fail(DECBPM_ERR_UNSUPPORTED, "Chebyshev degree on the PML spectrum too large (reduce dz)");
        J.assign(kmax + 1, 0.0);
        bessel_sequence(std::fabs(a), kmax, J.data());
        std::vector<double> tail(kmax + 2, 0.0);
        for (int k = kmax; k >= 0; --k) tail[k] = tail[k + 1] + 2.0 * std::fabs(J[k]) * std::pow(rho_e, k);
        M = 0;
        while (M < kmax && tail[M + 1] > tol) ++M;
        if (M < kmax - 20) break;
    }
    M = std::max(M, 2);
    out.coef.assign(M + 1, 0.0);
    for (int k = 0; k <= M; ++k) {
        const double jk = J[k] * ((a < 0 && (k & 1)) ? -1.0 : 1.0) * (k == 0 ? 1.0 : 2.0);
        out.coef[k] = std::pow(cd(0.0, -1.0), k) * jk;
    }
    out.c = c;
    out.r = r;
    out.M = M;
    out.theta0 = -dz * p1 * c;
    return DECBPM_OK;
}

template <typename R>
static int propagate_pml(decbpm_mesh_t m, const decbpm_params *prm, void *psi_dev, int64_t n_fields, cudaStream_t s,
                         decbpm_diag *diag_out) {
    using cd = std::complex<double>;
    using C = typename CT<R>::c2;
    if (prm->kerr_mode != DECBPM_KERR_LUMPED) return fail(DECBPM_ERR_UNSUPPORTED, "with a PML the split-step takes lumped Kerr");
    const int n0 = int(m->A.n0);
    PmlSeries ser;
    TRY(pml_series(m, prm->dz, default_tol(prm), ser));
    const double c = ser.c, r = ser.r, theta0 = ser.theta0;
    const int M = ser.M;
    const std::vector<cd> &coef = ser.coef;
    const R cs = R(c / r);
    // Stage table: b_k = a_k psi + 2 X~ b_{k+1} - b_{k+2}, the top two stages
    // folded (as in the march without a layer).  A constant field is mapped
    // exactly to -c' by the kernel's X~, so the lambda = 0 mode sees the
    // recurrence at x = -c' with the stored (rounded) coefficients: its FP64
    // value is set against the exact e^{-i theta0} through alpha_lo on the
    // last stage, leaving the smooth part of the field no systematic per-step
    // gain or phase error from coefficient rounding.
    auto mk = [](cd z) { C w; w.x = R(z.real()); w.y = R(z.imag()); return w; };   // host code: no cmk
    auto up = [](C z) { return cd(double(z.x), double(z.y)); };
    std::vector<PmlStage<R>> st(M);
    for (int k = M - 1; k >= 0; --k) {
        cd alpha = coef[k], beta = (k == 0) ? 1.0 : 2.0;
        int g_psi = 0, has_h = 1;
        if (k == M - 1) { g_psi = 1; beta = 2.0 * coef[M]; has_h = 0; }
        else if (k == M - 2) { alpha = coef[k] - coef[M]; has_h = 0; }
        st[k] = PmlStage<R>{mk(alpha), mk(beta), mk(0.0), g_psi, has_h, k == 0 ? 1 : 0};
    }
    {
        cd bk1 = 0, bk2 = 0, Sv = 0;
        const double x0 = -double(cs);
        for (int k = M - 1; k >= 0; --k) {
            const cd g = st[k].g_psi ? 1.0 : bk1;
            cd o = up(st[k].alpha) + up(st[k].beta) * (x0 * g);
            if (st[k].has_h) o -= bk2;
            if (k == 0) Sv = o;
            bk2 = bk1;
            bk1 = o;
        }
        st[0].alpha_lo = mk(std::exp(cd(0.0, -theta0)) - Sv);
    }
    decbpm_plan_t P = nullptr;
    TRY(single_plan(m, n_fields, prm->precision, &P));
    if (P->order.empty()) TRY(plan_configure<R>(P, prm->dz, default_tol(prm)));   // buffers and the device view
    PmlStepOps<R> po{};
    po.slice_ptr = m->slice_ptr; po.slice_w = m->slice_w; po.col = m->col;
    if constexpr (sizeof(R) == 4) {
        po.x = m->pml_x32; po.v = m->pml_v32; po.chib = m->pml_chib32; po.sigma = m->sig32;
    } else {
        po.x = m->pml_x64; po.v = m->pml_v; po.chib = m->pml_chib; po.sigma = m->sig64;
    }
    po.status = P->status;
    po.cs = cs;
    po.n0 = n0;
    po.bpad_log2 = P->bpad_log2;
    C *psi = (C *)P->psi[0];
    C *b[3] = {(C *)P->b0[0], (C *)P->b1[0], (C *)P->b2[0]};
    const int n_points = n_diag_points(prm);
    TRY(ensure_diag_host(P, n_points));
    const int64_t n_elem = int64_t(n0) << P->bpad_log2;
    if (n_elem > 0x7fffffff) return fail(DECBPM_ERR_UNSUPPORTED, "mesh x fields too large for the PML march");
    const int T = 256, G = int((n_elem + T - 1) / T);
    permute_in_kernel<C><<<std::min(G, 4 * P->num_sms), T, 0, s>>>((const C *)psi_dev, psi, m->perm, n0,
                                                                   int32_t(n_fields), P->bpad);
    const int64_t every = prm->diag_every > 0 ? prm->diag_every : std::max<int64_t>(prm->n_steps, 1);
    int point = 0;
    CK(cudaMemsetAsync(P->status, 0, sizeof(int), s));
    CK(cudaEventRecord(P->ev0, s));
    int pml_occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pml_occ, (const void *)pml_march_kernel<R>, 256, 0));
    const bool pml_fused = prm->variant != DECBPM_VARIANT_PLAIN && prm->n_steps > 0 && pml_occ >= 1 &&
                           int64_t(P->num_sms) * std::min(pml_occ, 6) * 256 >= n_elem;
    if (pml_fused) {
        // the stage table in the plan's PML workspace
        const size_t st_bytes = sizeof(PmlStage<R>) * size_t(M);
        if (st_bytes > P->pml_st_bytes) {
            TRY(P->mem.alloc(&P->pml_st, st_bytes));
            P->pml_st_bytes = st_bytes;
        }
        CK(cudaMemcpyAsync(P->pml_st, st.data(), st_bytes, cudaMemcpyHostToDevice, s));
        const int grid = std::min(P->num_sms * std::min(pml_occ, 6), std::max(1, G));
        for (int64_t done = 0; done < prm->n_steps;) {
            const int64_t nb = std::min<int64_t>(every, prm->n_steps - done);
            if (nb > 0x7fffffff) return fail(DECBPM_ERR_INVALID_ARG, "step block too long");
            PmlMarchParams<R> mp{};
            mp.o = po;
            mp.psi = psi;
            mp.b[0] = b[0]; mp.b[1] = b[1]; mp.b[2] = b[2];
            mp.st = reinterpret_cast<const PmlStage<R> *>(P->pml_st);
            mp.M = M;
            mp.n_steps = int32_t(nb);
            mp.pre_half = 1;
            mp.post_half = 1;
            mp.h = R(prm->dz);
            mp.barrier = P->barrier;
            mp.status = P->status;
            mp.timeout_ns = kBarrierTimeoutNs;
            CK(cudaMemsetAsync(P->barrier, 0, sizeof(unsigned long long), s));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(256);
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            void *args[] = {&mp};
            CK(cudaLaunchKernelExC(&cfg, (const void *)pml_march_kernel<R>, args));
            done += nb;
            if (done >= prm->n_steps) CK(cudaEventRecord(P->ev1, s));
            TRY(launch_diag<R>(P, s, DECBPM_KERR_LUMPED, point++));
        }
    }
    const R h = R(prm->dz), hh2 = R(0.5 * prm->dz);
    for (int64_t step = 0; step < prm->n_steps && !pml_fused; ++step) {
        const bool block_start = (step % every) == 0;
        const bool block_end = ((step + 1) % every) == 0 || step + 1 == prm->n_steps;
        if (block_start) pml_diag_kernel<R><<<G, T, 0, s>>>(po, psi, hh2);
        for (int k = M - 1; k >= 0; --k) {
            const C *g = st[k].g_psi ? psi : b[(k + 1) % 3];
            const C *hv = st[k].has_h ? b[(k + 2) % 3] : nullptr;
            C *outp = (k == 0) ? psi : b[k % 3];
            pml_stage_kernel<R><<<G, T, 0, s>>>(po, psi, g, hv, outp, st[k]);
        }
        pml_diag_kernel<R><<<G, T, 0, s>>>(po, psi, block_end ? hh2 : h);
        if (block_end) {
            if (step + 1 == prm->n_steps) CK(cudaEventRecord(P->ev1, s));
            TRY(launch_diag<R>(P, s, DECBPM_KERR_LUMPED, point++));
        }
    }
    if (prm->n_steps == 0) {
        CK(cudaEventRecord(P->ev1, s));
        TRY(launch_diag<R>(P, s, DECBPM_KERR_LUMPED, point++));
    }
    const double ph = std::fmod(double(prm->n_steps) * theta0, 2.0 * M_PI);
    permute_out_kernel<C><<<std::min(G, 4 * P->num_sms), T, 0, s>>>(psi, (C *)psi_dev, m->perm, n0, int32_t(n_fields),
                                                                    P->bpad, std::cos(ph), std::sin(ph));
    CK(cudaGetLastError());
    int status = 0;
    CK(cudaMemcpyAsync(&status, P->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (status == DECBPM_ERR_TIMEOUT) return fail(DECBPM_ERR_TIMEOUT, "grid barrier timed out in the PML march");
    if (status != 0) return fail(status, "device reported status %d", status);
    return finish_diag(P, prm, n_points, diag_out);
}

// ============================================================== C ABI
extern "C" {

#ifdef DECBPM_BOUNDS_CHECK
const char *decbpm_version(void) { return "decbpm 0.1 (sm_103a, bounds-checked)"; }
#else
const char *decbpm_version(void) { return "decbpm 0.1 (sm_103a)"; }
#endif

const char *decbpm_last_error(void) { return last_error_cstr(); }

int decbpm_assemble_host(const decbpm_mesh_desc *desc, decbpm_mesh_info_t *info, double *m, double *v, double *chib,
                         int64_t *K_rowptr, int32_t *K_col, double *K_val, int32_t *perm) {
    Assembly A;
    TRY(assemble(desc, A));
    Sell S;
    build_sell(A, S);
    if (info) {
        info->n_vertices = A.n0;
        info->n_edges = A.n_edges;
        info->n_cells = A.nc;
        info->nnz_offdiag = int64_t(A.col.size());
        info->max_degree = A.max_degree;
        info->n_p = int32_t(A.p.size());
        info->bandwidth = A.bandwidth;
        info->rho = A.rho;
        info->area = A.area;
        info->mean_degree = double(A.col.size()) / double(A.n0);
        info->sell_entries = int64_t(S.col.size());
        info->device_bytes = 0;
        info->rho_kind = A.rho_kind;
        info->pad_ = 0;
        info->rho_lanczos = A.rho_lanczos;
        info->rho_rigorous = A.rho_rigorous;
    }
    const int64_t n0 = A.n0;
    if (m) std::copy(A.m.begin(), A.m.end(), m);
    if (v) std::copy(A.v.begin(), A.v.end(), v);
    if (chib) std::copy(A.chib.begin(), A.chib.end(), chib);
    if (perm) std::copy(A.perm.begin(), A.perm.end(), perm);
    if (K_rowptr || K_col || K_val) {
        int64_t k = 0;
        for (int64_t p = 0; p < n0; ++p) {
            if (K_rowptr) K_rowptr[p] = k;
            bool diag_done = false;
            for (int64_t e = A.rowptr[p]; e <= A.rowptr[p + 1]; ++e) {
                const bool at_end = e == A.rowptr[p + 1];
                if (!diag_done && (at_end || A.col[e] > p)) {
                    if (K_col) K_col[k] = int32_t(p);
                    if (K_val) K_val[k] = A.wsum[p];
                    ++k;
                    diag_done = true;
                }
                if (at_end) break;
                if (K_col) K_col[k] = A.col[e];
                if (K_val) K_val[k] = -A.w[e];
                ++k;
            }
        }
        if (K_rowptr) K_rowptr[n0] = k;
    }
    return DECBPM_OK;
}

int decbpm_bessel_coefficients(double a, double tol, int32_t max_terms, double *J_out, int32_t *n_out) {
    if (!n_out || !(a >= 0) || !std::isfinite(a) || !(tol > 0)) return fail(DECBPM_ERR_INVALID_ARG, "bad arguments");
    Cheb cb;
    std::vector<double> p = {1.0};
    // a = h * p1 * r with rho = 2r; use h = a, r = 1
    TRY(cheb_coefficients(p, 2.0, a, tol, cb));
    const int n = cb.M + 1;
    *n_out = n;
    if (!J_out || max_terms < n) return fail(DECBPM_ERR_INVALID_ARG, "need %d terms", n);
    std::vector<double> J(n);
    bessel_sequence(a, n - 1, J.data());
    std::copy(J.begin(), J.end(), J_out);
    return DECBPM_OK;
}

int decbpm_mesh_create(const decbpm_mesh_desc *desc, decbpm_mesh_t *out) {
    NvtxRange nvtx_("decbpm_mesh_create");
    if (!out) return fail(DECBPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    auto M = std::make_unique<decbpm_mesh_s>();
    TRY(assemble(desc, M->A));
    {
        const int64_t nv = desc->n_vertices, nc = desc->n_cells;
        M->g_coords.assign(desc->coords, desc->coords + nv * desc->dim);
        M->g_cells.assign(desc->cells, desc->cells + nc * (desc->dim + 1));
        M->g_V.assign(nc, 0.0);
        M->g_chi.assign(nc, 1.0);
        if (desc->V_cell) M->g_V.assign(desc->V_cell, desc->V_cell + nc);
        if (desc->chi_cell) M->g_chi.assign(desc->chi_cell, desc->chi_cell + nc);
    }
    build_sell(M->A, M->S);
    CK(cudaGetDevice(&M->device));
    int rc = mesh_upload(M.get());
    if (rc != DECBPM_OK) {
        M->mem.release();
        return rc;
    }
    *out = M.release();
    return DECBPM_OK;
}

int decbpm_mesh_destroy(decbpm_mesh_t mesh) {
    if (!mesh) return DECBPM_OK;
    for (auto &p : mesh->plans) delete p.second;
    mesh->plans.clear();
    mesh->mem.release();
    delete mesh;
    return DECBPM_OK;
}

int decbpm_mesh_info(decbpm_mesh_t m, decbpm_mesh_info_t *info) {
    if (!m || !info) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    info->n_vertices = m->A.n0;
    info->n_edges = m->A.n_edges;
    info->n_cells = m->A.nc;
    info->nnz_offdiag = int64_t(m->A.col.size());
    info->max_degree = m->A.max_degree;
    info->n_p = int32_t(m->A.p.size());
    info->bandwidth = m->A.bandwidth;
    info->rho = m->A.rho;
    info->area = m->A.area;
    info->mean_degree = double(m->A.col.size()) / double(m->A.n0);
    info->sell_entries = int64_t(m->S.col.size());
    info->device_bytes = int64_t(m->mem.bytes);
    info->rho_kind = m->A.rho_kind;
    info->pad_ = 0;
    info->rho_lanczos = m->A.rho_lanczos;
    info->rho_rigorous = m->A.rho_rigorous;
    return DECBPM_OK;
}

static int single_plan(decbpm_mesh_t mesh, int64_t n_fields, int32_t precision, decbpm_plan_t *P,
                       bool field_groups) {
    if (n_fields < 1 || n_fields > kMaxFields) return fail(DECBPM_ERR_UNSUPPORTED, "n_fields must be in 1..%d", kMaxFields);
    // field groups (complex64, > kGroupFields fields) only for the forward
    // march's entry points; the adjoint, the PML march and the diagnostics
    // work on one entry
    field_groups = field_groups && precision == DECBPM_C64 && n_fields > kGroupFields;
    auto key = std::make_pair(int(n_fields), int(precision) | (field_groups ? 0x100 : 0));
    auto it = mesh->plans.find(key);
    if (it != mesh->plans.end()) { *P = it->second; return DECBPM_OK; }
    int32_t nf = int32_t(n_fields);
    TRY(plan_create_impl(&mesh, 1, &nf, precision, P, field_groups));
    mesh->plans[key] = *P;
    return DECBPM_OK;
}

int decbpm_propagate(decbpm_mesh_t mesh, const decbpm_params *params, void *psi_dev, int64_t n_fields, void *stream,
                     decbpm_diag *diag_out) {
    NvtxRange nvtx_("decbpm_propagate");
    clear_error();
    if (!mesh || !psi_dev) return fail(DECBPM_ERR_INVALID_ARG, "mesh and psi_dev are required");
    TRY(check_params(params));
    if (mesh->pml_on) {
        if (n_fields < 1) return fail(DECBPM_ERR_INVALID_ARG, "n_fields must be >= 1");
        return params->precision == DECBPM_C64
                   ? propagate_pml<float>(mesh, params, psi_dev, n_fields, (cudaStream_t)stream, diag_out)
                   : propagate_pml<double>(mesh, params, psi_dev, n_fields, (cudaStream_t)stream, diag_out);
    }
    if (params->variant == DECBPM_VARIANT_PLAIN) {
        if (n_fields != 1) return fail(DECBPM_ERR_UNSUPPORTED, "the plain variant runs one field");
        if (params->kerr_mode != DECBPM_KERR_LUMPED) return fail(DECBPM_ERR_UNSUPPORTED, "the plain variant runs lumped Kerr");
        return propagate_plain(mesh, params, psi_dev, (cudaStream_t)stream, diag_out);
    }
    decbpm_plan_t P;
    TRY(single_plan(mesh, n_fields, params->precision, &P, true));
    void *ptrs[1] = {psi_dev};
    return plan_propagate_dispatch(P, params, ptrs, stream, diag_out);
}

int decbpm_propagate_host(decbpm_mesh_t mesh, const decbpm_params *params, void *psi_host, int64_t n_fields, void *stream,
                          decbpm_diag *diag_out) {
    NvtxRange nvtx_("decbpm_propagate_host");
    clear_error();
    if (!mesh || !psi_host) return fail(DECBPM_ERR_INVALID_ARG, "mesh and psi_host are required");
    TRY(check_params(params));
    decbpm_plan_t P;
    // the staging buffer lives in the plan the march uses (the PML march runs one entry)
    TRY(single_plan(mesh, n_fields, params->precision, &P, !mesh->pml_on));
    const size_t bytes = size_t(mesh->A.n0) * n_fields * csize(params->precision);
    if (!P->user[0]) {
        char *t;
        TRY(P->mem.alloc(&t, bytes));
        P->user[0] = t;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(P->user[0], psi_host, bytes, cudaMemcpyHostToDevice, s));
    int rc;
    if (mesh->pml_on)
        rc = params->precision == DECBPM_C64 ? propagate_pml<float>(mesh, params, P->user[0], n_fields, s, diag_out)
                                             : propagate_pml<double>(mesh, params, P->user[0], n_fields, s, diag_out);
    else if (params->variant == DECBPM_VARIANT_PLAIN)
        rc = propagate_plain(mesh, params, P->user[0], s, diag_out);
    else
        rc = plan_propagate_dispatch(P, params, P->user.data(), stream, diag_out);
    if (rc != DECBPM_OK) return rc;
    CK(cudaMemcpyAsync(psi_host, P->user[0], bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return DECBPM_OK;
}

int decbpm_diagnostics(decbpm_mesh_t mesh, const void *psi_dev, int64_t n_fields, int32_t precision, void *stream,
                       decbpm_diag *diag_out) {
    clear_error();
    if (!mesh || !psi_dev || !diag_out) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    if (precision != DECBPM_C64 && precision != DECBPM_C128) return fail(DECBPM_ERR_INVALID_ARG, "bad precision");
    decbpm_plan_t P;
    TRY(single_plan(mesh, n_fields, precision, &P));
    cudaStream_t s = (cudaStream_t)stream;
    decbpm_params prm{};
    prm.dz = 1.0;
    prm.n_steps = 0;
    prm.precision = precision;
    TRY(ensure_diag_host(P, 1));
    const int64_t n0 = mesh->A.n0;
    const int blocks = int(std::min<int64_t>(4 * P->num_sms, (n0 * P->bpad + 255) / 256));
    if (precision == DECBPM_C64) {
        permute_in_kernel<float2><<<blocks, 256, 0, s>>>((const float2 *)psi_dev, (float2 *)P->psi[0], mesh->perm,
                                                         int32_t(n0), int32_t(n_fields), P->bpad);
        TRY(launch_diag<float>(P, s, DECBPM_KERR_LUMPED, 0));
    } else {
        permute_in_kernel<double2><<<blocks, 256, 0, s>>>((const double2 *)psi_dev, (double2 *)P->psi[0], mesh->perm,
                                                          int32_t(n0), int32_t(n_fields), P->bpad);
        TRY(launch_diag<double>(P, s, DECBPM_KERR_LUMPED, 0));
    }
    CK(cudaStreamSynchronize(s));
    return finish_diag(P, &prm, 1, diag_out);
}

int decbpm_plan_create(const decbpm_mesh_t *meshes, int32_t n_meshes, const int32_t *fields_per_mesh, int32_t precision,
                       decbpm_plan_t *out) {
    clear_error();
    return plan_create_impl(meshes, n_meshes, fields_per_mesh, precision, out, true);
}

int decbpm_plan_destroy(decbpm_plan_t plan) {
    delete plan;
    return DECBPM_OK;
}

int decbpm_plan_propagate(decbpm_plan_t plan, const decbpm_params *params, void *const *psi_dev, void *stream,
                          decbpm_diag *diag_out) {
    NvtxRange nvtx_("decbpm_plan_propagate");
    clear_error();
    return plan_propagate_dispatch(plan, params, psi_dev, stream, diag_out);
}

int decbpm_plan_propagate_host(decbpm_plan_t P, const decbpm_params *params, void *const *psi_host, void *stream,
                               decbpm_diag *diag_out) {
    NvtxRange nvtx_("decbpm_plan_propagate_host");
    clear_error();
    TRY(check_params(params));
    if (!P || !psi_host) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    TRY(reject_pml_plan(P));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t cs = csize(P->precision);
    for (size_t i = 0; i < P->user_meshes.size(); ++i) {
        if (!psi_host[i]) return fail(DECBPM_ERR_INVALID_ARG, "psi_host[%zu] is NULL", i);
        const size_t bytes = size_t(P->user_meshes[i]->A.n0) * P->user_B[i] * cs;
        if (!P->user[i]) {
            char *t;
            TRY(P->mem.alloc(&t, bytes));
            P->user[i] = t;
        }
        CK(cudaMemcpyAsync(P->user[i], psi_host[i], bytes, cudaMemcpyHostToDevice, s));
    }
    TRY(plan_propagate_dispatch(P, params, P->user.data(), stream, diag_out));
    for (size_t i = 0; i < P->user_meshes.size(); ++i) {
        const size_t bytes = size_t(P->user_meshes[i]->A.n0) * P->user_B[i] * cs;
        CK(cudaMemcpyAsync(psi_host[i], P->user[i], bytes, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return DECBPM_OK;
}

int32_t decbpm_plan_degree(decbpm_plan_t P, int32_t i, double dz, int32_t precision, double cheb_tol) {
    if (!P || i < 0 || i >= int32_t(P->user_meshes.size()) || !(dz > 0)) return 0;
    Cheb cb;
    const double tol = cheb_tol > 0 ? cheb_tol : (precision == DECBPM_C64 ? 1e-9 : 1e-16);
    const decbpm_mesh_t m = P->user_meshes[i];
    if (cheb_coefficients(m->A.p, m->A.rho, dz, tol, cb) != DECBPM_OK) return 0;
    return cb.M;
}

int decbpm_mesh_set_potential(decbpm_mesh_t m, const double *v_vertex) {
    clear_error();
    if (!m) return fail(DECBPM_ERR_INVALID_ARG, "mesh is NULL");
    const int64_t n0 = m->A.n0;
    std::vector<double> v(n0);
    for (int64_t i = 0; i < n0; ++i) {
        const int32_t o = m->A.perm[i];
        v[i] = v_vertex ? v_vertex[o] : m->A.v[o];
        if (!std::isfinite(v[i])) return fail(DECBPM_ERR_NONFINITE, "v_vertex[%d] is not finite", o);
    }
    std::vector<float> v32(v.begin(), v.end());
    CK(cudaMemcpy(m->vbase64, v.data(), sizeof(double) * n0, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->v64, v.data(), sizeof(double) * n0, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->v32, v32.data(), sizeof(float) * n0, cudaMemcpyHostToDevice));
    return DECBPM_OK;
}

int decbpm_mesh_set_potential_offset(decbpm_mesh_t m, const double *dv_dev, void *stream) {
    clear_error();
    if (!m) return fail(DECBPM_ERR_INVALID_ARG, "mesh is NULL");
    const int n0 = int(m->A.n0);
    potential_offset_kernel<<<(n0 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->vbase64, dv_dev, m->perm, m->v64,
                                                                              m->v32, n0);
    CK(cudaGetLastError());
    return DECBPM_OK;
}

int decbpm_vjp(decbpm_mesh_t mesh, const decbpm_params *params, const void *psi0_dev, const void *gN_dev,
               void *psiN_dev, void *grad_psi0_dev, double *grad_v_dev, int64_t n_fields, int32_t checkpoint_every,
               void *stream) {
    NvtxRange nvtx_("decbpm_vjp");
    clear_error();
    if (!mesh || !psi0_dev || !gN_dev || !grad_psi0_dev) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    TRY(reject_pml(mesh));
    TRY(check_params(params));
    if (params->kerr_mode != DECBPM_KERR_LUMPED) return fail(DECBPM_ERR_UNSUPPORTED, "the adjoint supports lumped Kerr");
    if (params->variant != DECBPM_VARIANT_FUSED) return fail(DECBPM_ERR_UNSUPPORTED, "the adjoint runs the fused variant");
    if (checkpoint_every < 0) return fail(DECBPM_ERR_INVALID_ARG, "checkpoint_every < 0");
    decbpm_plan_t P;
    TRY(single_plan(mesh, n_fields, params->precision, &P));
    cudaStream_t s = (cudaStream_t)stream;
    if (params->precision == DECBPM_C64)
        return vjp_impl<float>(mesh, P, params, psi0_dev, gN_dev, psiN_dev, grad_psi0_dev, grad_v_dev, n_fields,
                               checkpoint_every, s);
    return vjp_impl<double>(mesh, P, params, psi0_dev, gN_dev, psiN_dev, grad_psi0_dev, grad_v_dev, n_fields,
                            checkpoint_every, s);
}

int decbpm_adjoint(decbpm_mesh_t mesh, const decbpm_params *params, const void *psi0_dev, const void *target_dev,
                   int64_t n_fields, double *J_out, double *grad_v_dev, void *grad_psi0_dev, int32_t checkpoint_every,
                   void *stream) {
    NvtxRange nvtx_("decbpm_adjoint");
    clear_error();
    if (!mesh || !psi0_dev || !target_dev || !J_out) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    TRY(reject_pml(mesh));
    TRY(check_params(params));
    if (params->kerr_mode != DECBPM_KERR_LUMPED) return fail(DECBPM_ERR_UNSUPPORTED, "the adjoint supports lumped Kerr");
    if (params->variant != DECBPM_VARIANT_FUSED) return fail(DECBPM_ERR_UNSUPPORTED, "the adjoint runs the fused variant");
    if (checkpoint_every < 0) return fail(DECBPM_ERR_INVALID_ARG, "checkpoint_every < 0");
    decbpm_plan_t P;
    TRY(single_plan(mesh, n_fields, params->precision, &P));
    cudaStream_t s = (cudaStream_t)stream;
    if (params->precision == DECBPM_C64)
        return vjp_impl<float>(mesh, P, params, psi0_dev, nullptr, nullptr, grad_psi0_dev, grad_v_dev, n_fields,
                               checkpoint_every, s, target_dev, J_out);
    return vjp_impl<double>(mesh, P, params, psi0_dev, nullptr, nullptr, grad_psi0_dev, grad_v_dev, n_fields,
                            checkpoint_every, s, target_dev, J_out);
}

int decbpm_rk45(decbpm_mesh_t mesh, double z_end, int32_t kerr_mode, const decbpm_rk45_opts *opts, void *psi_dev,
                void *stream, decbpm_rk45_stats *stats) {
    NvtxRange nvtx_("decbpm_rk45");
    clear_error();
    if (!mesh || !opts || !psi_dev) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    if (!(z_end >= 0) || !std::isfinite(z_end)) return fail(DECBPM_ERR_INVALID_ARG, "z_end must be finite and >= 0");
    if (!(opts->rtol > 0) || !(opts->atol > 0)) return fail(DECBPM_ERR_INVALID_ARG, "rtol and atol must be > 0");
    if (kerr_mode != DECBPM_KERR_LUMPED && kerr_mode != DECBPM_KERR_ELEMENT) return fail(DECBPM_ERR_INVALID_ARG, "bad kerr_mode");
    if (mesh->pml_on && kerr_mode != DECBPM_KERR_LUMPED)
        return fail(DECBPM_ERR_UNSUPPORTED, "with a PML the RK45 path takes lumped Kerr");
    decbpm_plan_t P;
    TRY(single_plan(mesh, 1, DECBPM_C128, &P));
    if (P->order.empty()) TRY(plan_configure<double>(P, 1e-3, 1e-16));   // only for the device view of the mesh
    return rk45_impl(mesh, P, z_end, kerr_mode, opts, psi_dev, (cudaStream_t)stream, stats);
}

int decbpm_soliton(decbpm_mesh_t mesh, const decbpm_soliton_opts *opts, void *psi_dev, void *stream,
                   decbpm_soliton_stats *stats) {
    NvtxRange nvtx_("decbpm_soliton");
    clear_error();
    if (!mesh || !opts || !psi_dev) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    TRY(reject_pml(mesh));
    if (!(opts->power > 0) || !std::isfinite(opts->power)) return fail(DECBPM_ERR_INVALID_ARG, "power must be > 0");
    if (!(opts->tau > 0) || !std::isfinite(opts->tau)) return fail(DECBPM_ERR_INVALID_ARG, "tau must be > 0");
    if (!(opts->tol > 0)) return fail(DECBPM_ERR_INVALID_ARG, "tol must be > 0");
    if (opts->max_iter < 1) return fail(DECBPM_ERR_INVALID_ARG, "max_iter must be >= 1");
    if (!(opts->mix > 0) || opts->mix > 1) return fail(DECBPM_ERR_INVALID_ARG, "mix must be in (0, 1]");
    if (opts->kerr_mode != DECBPM_KERR_LUMPED && opts->kerr_mode != DECBPM_KERR_ELEMENT)
        return fail(DECBPM_ERR_INVALID_ARG, "bad kerr_mode");
    decbpm_plan_t P;
    TRY(single_plan(mesh, 1, DECBPM_C128, &P));
    if (P->order.empty()) TRY(plan_configure<double>(P, 1e-3, 1e-16));   // only for the device view of the mesh
    return soliton_impl(mesh, P, opts, psi_dev, (cudaStream_t)stream, stats);
}

int decbpm_bessel_i_scaled(double a, double tol, int32_t n_max, double *out, int32_t *n_out) {
    clear_error();
    if (!(a >= 0) || !std::isfinite(a) || !(tol > 0) || !n_out) return fail(DECBPM_ERR_INVALID_ARG, "bad argument");
    std::vector<double> sk;
    bessel_i_scaled(a, tol, sk);
    *n_out = int32_t(sk.size());
    if (out) for (int32_t k = 0; k < std::min<int32_t>(n_max, int32_t(sk.size())); ++k) out[k] = sk[k];
    return DECBPM_OK;
}

int decbpm_plan_autotune(decbpm_plan_t P, double dz, int32_t kerr_mode, int32_t trial_steps, void *stream,
                         decbpm_tune_result *out) {
    NvtxRange nvtx_("decbpm_plan_autotune");
    clear_error();
    if (!P) return fail(DECBPM_ERR_INVALID_ARG, "plan is NULL");
    TRY(reject_pml_plan(P));
    if (!(dz > 0) || !std::isfinite(dz)) return fail(DECBPM_ERR_INVALID_ARG, "dz must be finite and > 0");
    if (trial_steps < 1 || trial_steps > 1000) return fail(DECBPM_ERR_INVALID_ARG, "trial_steps must be in 1..1000");
    if (kerr_mode != DECBPM_KERR_LUMPED && kerr_mode != DECBPM_KERR_ELEMENT) return fail(DECBPM_ERR_INVALID_ARG, "bad kerr_mode");
    if (P->precision == DECBPM_C64) return autotune_impl<float>(P, dz, kerr_mode, trial_steps, (cudaStream_t)stream, out);
    return autotune_impl<double>(P, dz, kerr_mode, trial_steps, (cudaStream_t)stream, out);
}

int decbpm_plan_set_shape(decbpm_plan_t P, const decbpm_tune_result *shape) {
    clear_error();
    if (!P || !shape) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    TuneChoice c{};
    c.forward = shape->forward_walk ? 1 : 0;
    c.fpt = shape->values_per_thread > 0 ? shape->values_per_thread : default_fpt(P->precision, P->bpad);
    if (shape->variant == DECBPM_VARIANT_PAIRS) {
        if (!P->pair_mode) return fail(DECBPM_ERR_UNSUPPORTED, "this plan cannot run the stage-pair kernel");
        if (shape->tile_slots < 2 || shape->tile_slots > P->pair_slots)
            return fail(DECBPM_ERR_INVALID_ARG, "tile_slots must be in 2..%d", P->pair_slots);
        c.pair = 1; c.per_sm = 1; c.slots = shape->tile_slots;
        c.fpt = default_fpt(P->precision, P->bpad);
    } else if (shape->variant == DECBPM_VARIANT_FUSED || shape->variant == DECBPM_VARIANT_FLOW) {
        if (!P->tile_mode) return fail(DECBPM_ERR_UNSUPPORTED, "this plan cannot run the tile-staged kernel");
        if (shape->variant == DECBPM_VARIANT_FLOW && !P->flow_mode)
            return fail(DECBPM_ERR_UNSUPPORTED, "this plan cannot run the dataflow kernel");
        if (shape->tile_slots < 2 || shape->tile_slots > P->n_slots)
            return fail(DECBPM_ERR_INVALID_ARG, "tile_slots must be in 2..%d", P->n_slots);
        if (shape->variant == DECBPM_VARIANT_FLOW && (shape->walk_skip < 0 || shape->walk_skip > 4096))
            return fail(DECBPM_ERR_INVALID_ARG, "walk_skip must be in 0..4096");
        c.slots = shape->tile_slots; c.per_sm = P->max_per_sm;
        c.fpt = default_fpt(P->precision, P->bpad);
        c.flow = shape->variant == DECBPM_VARIANT_FLOW ? 1 : 0;
        c.skip = c.flow ? (shape->walk_skip > 0 ? shape->walk_skip : kDefaultFlowSkip) : 0;
        c.ranges = c.flow && shape->flow_ranges ? 1 : 0;
    } else if (shape->variant == DECBPM_VARIANT_ROWS) {
        if (!fpt_allowed(P->precision, P->bpad, c.fpt))
            return fail(DECBPM_ERR_UNSUPPORTED, "values_per_thread %d is not built for this plan", c.fpt);
        int occ = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, march_kernel_ptr(P->precision, P->bpad, c.fpt), P->block, 0));
        if (shape->ctas_per_sm < 1 || shape->ctas_per_sm > std::min(occ, 4))
            return fail(DECBPM_ERR_INVALID_ARG, "ctas_per_sm must be in 1..%d", std::min(occ, 4));
        c.rows = 1; c.per_sm = shape->ctas_per_sm;
        c.nometa = shape->no_meta_cache ? 1 : 0;
    } else {
        return fail(DECBPM_ERR_INVALID_ARG, "bad variant %d", shape->variant);
    }
    apply_choice(P, c);
    return DECBPM_OK;
}

int decbpm_mesh_set_pml(decbpm_mesh_t mesh, const decbpm_pml *pml) {
    NvtxRange nvtx_("decbpm_mesh_set_pml");
    clear_error();
    if (!mesh) return fail(DECBPM_ERR_INVALID_ARG, "mesh is NULL");
    if (!pml || pml->sigma_max == 0.0) {
        mesh->pml_on = false;
        return DECBPM_OK;
    }
    return set_pml_impl(mesh, pml);
}

int32_t decbpm_mesh_pml_degree(decbpm_mesh_t mesh, double dz, int32_t precision, double cheb_tol) {
    if (!mesh || !mesh->pml_on || !(dz > 0) || !std::isfinite(dz)) return 0;
    if (precision != DECBPM_C64 && precision != DECBPM_C128) return 0;
    decbpm_params prm{};
    prm.dz = dz;
    prm.precision = precision;
    prm.cheb_tol = cheb_tol;
    PmlSeries ser;
    if (pml_series(mesh, dz, default_tol(&prm), ser) != DECBPM_OK) return 0;
    return ser.M;
}

int decbpm_plan_get_config(decbpm_plan_t P, decbpm_plan_config *cfg) {
    if (!P || !cfg) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    cfg->grid = P->grid;
    cfg->block = P->block;
    cfg->fields_padded = P->bpad;
    cfg->graphs = (P->graphs_ok && !P->graphs.empty()) ? 1 : 0;
    cfg->stages = P->S;
    cfg->n_meshes = int32_t(P->user_meshes.size());
    cfg->field_groups = int32_t(P->meshes.size());
    cfg->tile_slots = P->tile_mode ? P->n_slots : 0;
    cfg->tile_slot_bytes = P->tile_mode ? P->slot_bytes : 0;
    cfg->tile_grid = P->tile_mode ? P->tile_grid : 0;
    cfg->tile_block = P->tile_mode ? kTileThreads : 0;
    cfg->tuned = P->tuned ? 1 : 0;
    cfg->fused_kernel = (P->tile_mode && !P->tune_rows) ? 1 : 0;
    cfg->tile_slots_used =
        (P->tile_mode && !P->tune_rows) ? (P->tune_slots > 0 ? std::min(P->tune_slots, P->n_slots) : P->n_slots) : 0;
    cfg->forward_walk = P->forward_walk;
    if (cfg->fused_kernel == 1 && P->pair_mode && P->tune_pair == 1) {
        cfg->fused_kernel = 2;
        cfg->tile_slots_used = P->tune_slots > 0 ? std::min(P->tune_slots, P->pair_slots) : P->pair_slots;
    } else if (cfg->fused_kernel == 1 && P->flow_mode && P->tune_flow == 1) {
        cfg->fused_kernel = 3;
    }
    cfg->tile_rows = P->tile_mode ? (P->tile_one ? kTile1Rows : kTileRows) : 0;
    cfg->flow_grid = P->flow_mode ? P->flow_grid : 0;
    cfg->flow_skip = P->flow_skip;
    cfg->flow_ranges = P->flow_ranges;
    cfg->meta_items = 0;
    if (cfg->fused_kernel == 0) {
        const void *fn = march_kernel_ptr(P->precision, P->bpad, P->fpt);
        cfg->meta_items = row_meta_cache(P, fn, P->grid, P->fpt).first;
    }
    cfg->pair_slots = P->pair_mode ? P->pair_slots : 0;
    cfg->pair_slot_bytes = P->pair_mode ? P->pair_slot_bytes : 0;
    cfg->pair_grid = P->pair_mode ? P->pair_grid : 0;
    cfg->passes = P->pair_mode ? P->n_passes : 0;
    cfg->values_per_thread = P->fpt;
    cfg->rows_per_item = 32 * P->fpt / P->bpad;
    return DECBPM_OK;
}

int decbpm_plan_last_march_ms(decbpm_plan_t P, double *ms) {
    if (!P || !ms) return fail(DECBPM_ERR_INVALID_ARG, "NULL argument");
    float t = 0;
    CK(cudaEventElapsedTime(&t, P->ev0, P->ev1));
    *ms = double(t);
    return DECBPM_OK;
}

int decbpm_selftest_barrier(int32_t missing_arrivals, int64_t timeout_ns, void *stream) {
    clear_error();
    if (missing_arrivals < 0 || timeout_ns <= 0 || timeout_ns > 10000000000LL)
        return fail(DECBPM_ERR_INVALID_ARG, "missing_arrivals >= 0 and 0 < timeout_ns <= 1e10 required");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *bar = nullptr;
    int *status = nullptr;
    CK(cudaMalloc(&bar, sizeof(unsigned long long)));
    CK(cudaMalloc(&status, sizeof(int)));
    CK(cudaMemsetAsync(bar, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(status, 0, sizeof(int), s));
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(sms, 8));
    cfg.blockDim = dim3(64);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    long long tns = timeout_ns;
    unsigned extra = unsigned(missing_arrivals);
    cudaError_t e = cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, bar, status, tns, extra);
    int st = 0;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bar);
    cudaFree(status);
    if (e != cudaSuccess) return fail(DECBPM_ERR_CUDA, "self test: %s", cudaGetErrorString(e));
    if (st == DECBPM_ERR_TIMEOUT) return fail(DECBPM_ERR_TIMEOUT, "barrier wait ran out (as requested)");
    return st;
}

int decbpm_selftest_bounds_check(void *stream) {
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    int *buf = nullptr;                       // [status, returned index]
    CK(cudaMalloc(&buf, 2 * sizeof(int)));
    cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), s);
    const int n = 1000;
    if (e == cudaSuccess) {
        index_check_selftest_kernel<<<1, 32, 0, s>>>(n, buf, buf + 1);
        e = cudaGetLastError();
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(h, buf, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(DECBPM_ERR_CUDA, "self test: %s", cudaGetErrorString(e));
#ifdef DECBPM_BOUNDS_CHECK
    if (h[0] != DECBPM_ERR_DEVICE_CHECK || h[1] != 0)
        return fail(DECBPM_ERR_CUDA, "index check did not fire (status %d, index %d)", h[0], h[1]);
    return fail(DECBPM_ERR_DEVICE_CHECK, "index %d of a %d-element buffer reported (as requested)", n, n);
#else
    if (h[0] != 0 || h[1] != n) return fail(DECBPM_ERR_CUDA, "unexpected status %d, index %d", h[0], h[1]);
    return DECBPM_OK;
#endif
}

int decbpm_propagate_batch(const decbpm_mesh_t *meshes, int32_t n_meshes, const int32_t *fields_per_mesh,
                           const decbpm_params *params, void *const *psi_dev, void *stream, decbpm_diag *diag_out) {
    NvtxRange nvtx_("decbpm_propagate_batch");
    clear_error();
    TRY(check_params(params));
    decbpm_plan_t P = nullptr;
    TRY(plan_create_impl(meshes, n_meshes, fields_per_mesh, params->precision, &P, true));
    if (P->meshes.size() && reject_pml_plan(P) != DECBPM_OK) { delete P; return DECBPM_ERR_UNSUPPORTED; }
    int rc = plan_propagate_dispatch(P, params, psi_dev, stream, diag_out);
    delete P;
    return rc;
}

}  // extern "C"

// ============================================================== allocation-free propagate
// Some callers cannot allocate device memory at the point where they want to
// propagate: code running while a framework's caching allocator owns the
// whole memory budget, or loops that must keep a fixed memory footprint.
// For them, decbpm_propagate_noalloc keeps its scratch (the internal-order
// copy of the field, the three Clenshaw buffers, the stage tables and the
// barrier/status words) in the file-scope device array below instead of in
// cudaMalloc'ed workspaces.  Every GPU that loads this library holds the
// array until the process exits.
constexpr size_t kNoallocScratchBytes = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {
struct NoallocSlot {
    bool ready = false;
    unsigned char *base = nullptr;
};
constexpr int kNoallocMaxDevices = 64;
NoallocSlot g_noalloc_slot[kNoallocMaxDevices];
std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and kept for the process; a
// cudaDeviceReset unloads the module and leaves the kept address stale (the
// header tells callers not to use this entry point after a reset).
int noalloc_scratch_base(int dev, unsigned char **base) {
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(DECBPM_ERR_UNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot &sl = g_noalloc_slot[dev];
    if (!sl.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(DECBPM_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s", cudaGetErrorString(e));
        sl.base = static_cast<unsigned char *>(p);
        sl.ready = true;
    }
    *base = sl.base;
    return DECBPM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename R>
int propagate_noalloc_impl(decbpm_mesh_t mesh, const decbpm_params *prm, void *psi_dev, int64_t n_fields,
                           cudaStream_t s) {
    using C = typename CT<R>::c2;
    const int64_t n0 = mesh->A.n0;
    const int bpad_log2 = ilog2(int(n_fields));
    const int bpad = 1 << bpad_log2;
    const int fpt = sizeof(R) == 4 ? std::min(bpad, DECBPM_FPT4) : (bpad > 32 ? 2 : 1);
    Cheb cb;
    TRY(cheb_coefficients(mesh->A.p, mesh->A.rho, prm->dz, default_tol(prm), cb));
    const int M = cb.M;
    // scratch layout: [barrier u64, status int] [view] [coef[M]] [active[M]] [psi] [b0] [b1] [b2]
    const size_t state = align256(size_t(n0) * bpad * sizeof(C));
    const size_t off_view = 256;
    const size_t off_coef = off_view + align256(sizeof(MeshView<R>));
    const size_t off_active = off_coef + align256(sizeof(StageCoef<R>) * M);
    const size_t off_psi = off_active + align256(sizeof(int32_t) * M);
    const size_t need = off_psi + 4 * state;
    if (need > kNoallocScratchBytes)
        return fail(DECBPM_ERR_INVALID_ARG,
                    "decbpm_propagate_noalloc needs %zu bytes of scratch for %lld vertices x %d padded fields "
                    "(degree %d) but its static scratch holds %zu bytes; use decbpm_propagate",
                    need, (long long)n0, bpad, M, kNoallocScratchBytes);
    int dev = 0, sms = 0, per_sm = 0;
    CK(cudaGetDevice(&dev));
    if (dev != mesh->device)
        return fail(DECBPM_ERR_INVALID_ARG, "the mesh lives on device %d but device %d is current", mesh->device, dev);
    unsigned char *base = nullptr;
    TRY(noalloc_scratch_base(dev, &base));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, march_ptr_for<R>(bpad), 256, 0));
    if (per_sm < 1) return fail(DECBPM_ERR_CUDA, "march kernel cannot be resident");
    C *psi = reinterpret_cast<C *>(base + off_psi);
    C *b[3] = {reinterpret_cast<C *>(base + off_psi + state), reinterpret_cast<C *>(base + off_psi + 2 * state),
               reinterpret_cast<C *>(base + off_psi + 3 * state)};
    // stage table, same recurrence and lambda = 0 residual as the plans
    StageCoef<R> coef[1024];
    if (M > 1024) return fail(DECBPM_ERR_UNSUPPORTED, "Chebyshev degree %d above 1024 (reduce dz)", M);
    auto mk = [](std::complex<double> z) { C c; c.x = R(z.real()); c.y = R(z.imag()); return c; };
    for (int k = 0; k < M; ++k) {
        StageCoef<R> sc{};
        std::complex<double> alpha = cb.a[k], beta = (k == 0) ? 1.0 : 2.0;
        int flags = 0;
        if (k == M - 1) { flags |= kGisPsi; beta = 2.0 * cb.a[M]; }
        else if (k == M - 2) { alpha = cb.a[k] - cb.a[M]; }
        else flags |= kHasH;
        if (k == 0) flags |= kFinal;
        sc.alpha = mk(alpha);
        sc.beta = mk(beta);
        sc.alpha_lo = mk(0.0);
        sc.flags = flags;
        coef[k] = sc;
    }
    {
        auto up = [](C z) { return std::complex<double>(double(z.x), double(z.y)); };
        std::complex<double> bk1 = 0, bk2 = 0, Sv = 0;
        for (int k = M - 1; k >= 0; --k) {
            const std::complex<double> g = (coef[k].flags & kGisPsi) ? 1.0 : bk1;
            std::complex<double> o = up(coef[k].alpha) - up(coef[k].beta) * g;
            if (coef[k].flags & kHasH) o -= bk2;
            if (coef[k].flags & kFinal) Sv = o;
            bk2 = bk1;
            bk1 = o;
        }
        coef[0].alpha_lo = mk(cb.f0 - Sv);
    }
    const int tpr_log2 = bpad_log2 - (fpt == 8 ? 3 : fpt == 4 ? 2 : fpt == 2 ? 1 : 0);
    const int rpw = 32 >> tpr_log2;
    const int items = int((n0 + rpw - 1) / rpw);
    int32_t active[1024];
    for (int k = 0; k < M; ++k) active[k] = items;
    MeshView<R> v{};
    v.n0 = int32_t(n0);
    v.n_slices = int32_t(mesh->S.n_slices);
    v.M = M;
    v.item_begin = 0;
    v.slice_ptr = mesh->slice_ptr; v.slice_w = mesh->slice_w; v.col = mesh->col;
    if constexpr (sizeof(R) == 4) {
        v.xval = mesh->x32; v.v = mesh->v32; v.chib = mesh->chib32; v.sigma = mesh->sig32;
        v.coff = mesh->coff32; v.cdiag = mesh->cdiag32;
    } else {
        v.xval = mesh->x64; v.v = mesh->v64; v.chib = mesh->chib64; v.sigma = mesh->sig64;
        v.coff = mesh->coff64; v.cdiag = mesh->cdiag64;
    }
    v.psi = psi; v.b[0] = b[0]; v.b[1] = b[1]; v.b[2] = b[2];
    v.coef = reinterpret_cast<const StageCoef<R> *>(base + off_coef);
    // the array keeps the previous call's contents: clear the barrier and status words
    CK(cudaMemsetAsync(base, 0, 256, s));
    CK(cudaMemcpyAsync(base + off_view, &v, sizeof(v), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + off_coef, coef, sizeof(StageCoef<R>) * M, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(base + off_active, active, sizeof(int32_t) * M, cudaMemcpyHostToDevice, s));
    const int pblocks = int(std::min<int64_t>(4 * sms, (n0 * bpad + 255) / 256));
    permute_in_kernel<C><<<pblocks, 256, 0, s>>>((const C *)psi_dev, psi, mesh->perm, int32_t(n0), int32_t(n_fields), bpad);
    CK(cudaGetLastError());
    if (prm->n_steps > 0) {
        if (prm->n_steps > 0x7fffffff) return fail(DECBPM_ERR_INVALID_ARG, "n_steps too large");
        MarchParams<R> mp{};
        mp.meshes = reinterpret_cast<const MeshView<R> *>(base + off_view);
        mp.active_items = reinterpret_cast<const int32_t *>(base + off_active);
        mp.n_meshes = 1;
        mp.S = M;
        mp.total_items = items;
        mp.n_steps = int32_t(prm->n_steps);
        mp.pre_half = 1;
        mp.post_half = 1;
        mp.kerr_mode = prm->kerr_mode;
        mp.bpad_log2 = bpad_log2;
        mp.h = R(prm->dz);
        mp.barrier = reinterpret_cast<unsigned long long *>(base);
        mp.status = reinterpret_cast<int *>(base + 8);
        mp.timeout_ns = kBarrierTimeoutNs;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(sms * std::min(per_sm, 4));
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void *args[] = {&mp};
        CK(cudaLaunchKernelExC(&cfg, march_ptr_for<R>(bpad), args));
    }
    const double ph = std::fmod(double(prm->n_steps) * cb.theta0, 2.0 * M_PI);
    const int oblocks = int(std::min<int64_t>(4 * sms, (n0 * n_fields + 255) / 256));
    permute_out_kernel<C><<<oblocks, 256, 0, s>>>(psi, (C *)psi_dev, mesh->perm, int32_t(n0), int32_t(n_fields), bpad,
                                                 std::cos(ph), std::sin(ph));
    CK(cudaGetLastError());
    int status = 0;
    CK(cudaMemcpyAsync(&status, base + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (status == DECBPM_ERR_TIMEOUT) return fail(DECBPM_ERR_TIMEOUT, "grid barrier timed out in the march kernel");
    if (status != 0) return fail(status, "device reported status %d", status);
    return DECBPM_OK;
}
}  // namespace

extern "C" int decbpm_propagate_noalloc(decbpm_mesh_t mesh, const decbpm_params *params, void *psi_dev,
                                        int64_t n_fields, void *stream) {
    NvtxRange nvtx_("decbpm_propagate_noalloc");
    clear_error();
    if (!mesh || !psi_dev) return fail(DECBPM_ERR_INVALID_ARG, "mesh and psi_dev are required");
    TRY(check_params(params));
    if (params->variant != DECBPM_VARIANT_FUSED)
        return fail(DECBPM_ERR_UNSUPPORTED, "decbpm_propagate_noalloc runs the fused variant only");
    TRY(reject_pml(mesh));
    if (n_fields < 1 || n_fields > kMaxFields) return fail(DECBPM_ERR_UNSUPPORTED, "n_fields must be in 1..%d", kMaxFields);
    cudaStream_t s = (cudaStream_t)stream;
    if (params->precision == DECBPM_C64) return propagate_noalloc_impl<float>(mesh, params, psi_dev, n_fields, s);
    return propagate_noalloc_impl<double>(mesh, params, psi_dev, n_fields, s);
}
