// Host-side algorithms of libvie: voxel/face mesh of an atom type, grid
// hierarchy and far-block lists, the greedy least-loaded work map and the
// work lists of the compressed apply.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <map>
#include <numeric>
#include <queue>

#include "common.h"

namespace vie {

std::atomic<long long> g_kernel_launches{0};

void fail(int status, const std::string& msg) { throw Error{status, msg}; }

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static thread_local Ctx* t_alloc_ctx = nullptr;

AllocScope::AllocScope(Ctx* c) : prev(t_alloc_ctx) { t_alloc_ctx = c; }
AllocScope::~AllocScope() { t_alloc_ctx = prev; }

void DevBuf::alloc(size_t b) {
    release();
    if (b == 0) b = 1;
    Ctx* c = t_alloc_ctx;
    if (c) {
        const int64_t cap = c->cap.load();
        const int64_t now = c->allocated.fetch_add((int64_t)b) + (int64_t)b;
        if (cap > 0 && now > cap) {
            c->allocated.fetch_sub((int64_t)b);
            fail(VIE_ERR_OOM, "allocation of " + std::to_string(b) + " bytes would exceed the context's cap of " +
                                  std::to_string(cap) + " bytes");
        }
    }
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        if (c) c->allocated.fetch_sub((int64_t)b);
        cudaGetLastError();
        fail(VIE_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = b;
    owner = c;
    if (c) {
        int64_t pk = c->peak.load(), cur = c->allocated.load();
        while (cur > pk && !c->peak.compare_exchange_weak(pk, cur)) {
        }
    }
}

void DevBuf::release() {
    if (p) {
        cudaFree(p);
        if (owner) owner->allocated.fetch_sub((int64_t)bytes);
    }
    p = nullptr;
    bytes = 0;
    owner = nullptr;
}

// ---------------------------------------------------------------------------
// Sec. 3 basis on a voxelised cube: one rooftop per voxel face.  Faces are
// numbered x-faces, y-faces, z-faces; inside a direction lexicographically in
// (i, j, k) with the normal index running 0..nv.
// ---------------------------------------------------------------------------
MeshTables build_mesh(double side, int nv) {
    MeshTables m;
    m.nv = nv;
    m.side = side;
    m.h = side / nv;
    m.nvox = nv * nv * nv;
    auto vnum = [nv](int i, int j, int k) { return (i * nv + j) * nv + k; };
    for (int i = 0; i < nv; ++i)
        for (int j = 0; j < nv; ++j)
            for (int k = 0; k < nv; ++k) {
                m.vox_ijk.push_back(i);
                m.vox_ijk.push_back(j);
                m.vox_ijk.push_back(k);
            }
    for (int d = 0; d < 3; ++d) {
        int ext[3] = {nv, nv, nv};
        ext[d] = nv + 1;
        for (int i = 0; i < ext[0]; ++i)
            for (int j = 0; j < ext[1]; ++j)
                for (int k = 0; k < ext[2]; ++k) {
                    int ijk[3] = {i, j, k};
                    int mm = ijk[d];
                    int f = (int)m.face_dir.size();
                    m.face_dir.push_back(d);
                    int below[3] = {i, j, k};
                    below[d] = mm - 1;
                    m.face_lo.push_back(mm >= 1 ? vnum(below[0], below[1], below[2]) : -1);
                    m.face_hi.push_back(mm <= nv - 1 ? vnum(i, j, k) : -1);
                    if (mm == 0 || mm == nv) {
                        m.face_sheet.push_back((int)m.surf_face.size());
                        m.face_sheet_sign.push_back(mm == 0 ? +1 : -1);
                        m.surf_face.push_back(f);
                    } else {
                        m.face_sheet.push_back(-1);
                        m.face_sheet_sign.push_back(0);
                    }
                }
    }
    m.np = (int)m.face_dir.size();
    m.nsurf = (int)m.surf_face.size();
    return m;
}

// ---------------------------------------------------------------------------
// Grid hierarchy (Sec. 5.1 Definition, Sec. 5.3 eq. eq_rec01, Sec. 5.4).
// Power-of-two quadtree over a root square of side s 2^L whose finest boxes
// (side s = smallest infinity-norm centre separation) hold at most one atom.
// Blocks are listed by level, then target box (y, x), then source box (y, x).
// ---------------------------------------------------------------------------
void build_tree(Op& op) {
    const int N = op.N;
    op.blocks.clear();
    op.block_atoms.clear();
    if (N == 1) {
        op.L = 0;
        return;
    }
    std::vector<double> x(N), y(N);
    for (int a = 0; a < N; ++a) {
        x[a] = op.centres[3 * a];
        y[a] = op.centres[3 * a + 1];
    }
    double s = std::numeric_limits<double>::infinity();
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) s = std::min(s, std::max(std::fabs(x[a] - x[b]), std::fabs(y[a] - y[b])));
    if (!(s > 0)) fail(VIE_ERR_INVALID_ARG, "two atoms share the same (x, y) position");
    double xmin = *std::min_element(x.begin(), x.end()), xmax = *std::max_element(x.begin(), x.end());
    double ymin = *std::min_element(y.begin(), y.end()), ymax = *std::max_element(y.begin(), y.end());
    double ext = std::max(xmax - xmin, ymax - ymin);
    int L = 0;
    while (std::ldexp(1.0, L) < ext / s + 1.0 - 1e-9) ++L;
    if (L > 20) fail(VIE_ERR_INVALID_ARG, "atom layout needs more than 20 grid levels");
    op.L = L;
    const long long side_boxes = 1LL << L;
    std::vector<long long> fx(N), fy(N);
    for (int a = 0; a < N; ++a) {
        fx[a] = std::min(side_boxes - 1, std::max(0LL, (long long)std::floor((x[a] - (xmin - 0.5 * s)) / s)));
        fy[a] = std::min(side_boxes - 1, std::max(0LL, (long long)std::floor((y[a] - (ymin - 0.5 * s)) / s)));
    }
    for (int lev = 1; lev <= L; ++lev) {
        int shift = L - lev;
        std::map<std::pair<long long, long long>, std::vector<int>> boxes;  // key (y, x), sorted
        for (int a = 0; a < N; ++a) boxes[{fy[a] >> shift, fx[a] >> shift}].push_back(a);
        for (auto& tb : boxes) {
            long long ty = tb.first.first, tx = tb.first.second;
            // candidate source boxes: children of the 3x3 parent neighbourhood
            std::vector<std::pair<long long, long long>> cand;
            for (long long py = (ty >> 1) - 1; py <= (ty >> 1) + 1; ++py)
                for (long long px = (tx >> 1) - 1; px <= (tx >> 1) + 1; ++px)
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            std::pair<long long, long long> key{2 * py + cy, 2 * px + cx};
                            if (py >= 0 && px >= 0 && boxes.count(key)) cand.push_back(key);
                        }
            std::sort(cand.begin(), cand.end());
            for (auto& key : cand) {
                long long dist = std::max(std::llabs(key.first - ty), std::llabs(key.second - tx));
                bool far = (lev == L) ? (dist != 0) : (dist > 1);
                if (!far) continue;
                const auto& ta = tb.second;
                const auto& sa = boxes[key];
                FarBlock b;
                b.level = lev;
                b.nt = (int)ta.size();
                b.ns = (int)sa.size();
                b.t_off = (int)op.block_atoms.size();
                op.block_atoms.insert(op.block_atoms.end(), ta.begin(), ta.end());
                b.s_off = (int)op.block_atoms.size();
                op.block_atoms.insert(op.block_atoms.end(), sa.begin(), sa.end());
                b.m = b.nt * op.np;
                b.n = b.ns * op.np;
                b.dist = (int)dist;
                b.dmin = (int)std::min(std::llabs(key.first - ty), std::llabs(key.second - tx));
                op.blocks.push_back(b);
            }
        }
    }
    // pair every block with its mirror (the far relation is symmetric)
    std::map<std::tuple<int, int, int>, int> idx;
    for (size_t i = 0; i < op.blocks.size(); ++i) {
        const auto& b = op.blocks[i];
        idx[{b.level, op.block_atoms[b.t_off], op.block_atoms[b.s_off]}] = (int)i;
    }
    for (size_t i = 0; i < op.blocks.size(); ++i) {
        auto& b = op.blocks[i];
        auto it = idx.find({b.level, op.block_atoms[b.s_off], op.block_atoms[b.t_off]});
        if (it == idx.end()) fail(VIE_ERR_STATE, "far block without a mirror");
        b.mirror = it->second;
    }
}

// ---------------------------------------------------------------------------
// App. C: greedy least-loaded assignment.  Interactions sorted by decreasing
// weight are given one by one to the currently least-loaded process (lowest
// index on ties).
// ---------------------------------------------------------------------------
void lpt_assign(const std::vector<double>& w, int nproc, std::vector<int>& owner, std::vector<double>& loads) {
    std::vector<int> order(w.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
    using E = std::pair<double, int>;
    std::priority_queue<E, std::vector<E>, std::greater<E>> heap;
    for (int k = 0; k < nproc; ++k) heap.push({0.0, k});
    owner.assign(w.size(), 0);
    loads.assign(nproc, 0.0);
    for (int i : order) {
        E top = heap.top();
        heap.pop();
        owner[i] = top.second;
        loads[top.second] += w[i];
        heap.push({loads[top.second], top.second});
    }
}

// ---------------------------------------------------------------------------
// Work lists of the compressed apply (see apply.cu for the item layouts).
//  phase 1 (t = R x): item (block, k0, k1): rows k0..k1 of R_b
//  phase 2 (F = sum Q t): item (atom, p0, p1): rows p0..p1 of that atom,
//          looping over the blocks whose target box holds the atom
// Items are mapped to persistent CTAs with the greedy least-loaded rule,
// weighted by their factor bytes.
// ---------------------------------------------------------------------------
static void pack_lpt(const std::vector<int4>& items, const std::vector<double>& w, int ncta,
                     std::vector<int4>& out_items, std::vector<int>& cta_ptr, std::vector<int>* perm = nullptr,
                     const std::vector<uint64_t>* key = nullptr) {
    std::vector<int> owner;
    std::vector<double> loads;
    lpt_assign(w, ncta, owner, loads);
    std::vector<std::vector<int>> per(ncta);
    // within a CTA keep the heaviest items first, or, given a spatial key, the
    // items in key order: every CTA then sweeps the array in the same
    // direction at about the same pace (its items' weights are spread evenly
    // over the keys), so the vector rows the CTAs gather at any one time come
    // from one region and stay in L2 (the order inside a CTA does not change
    // its load)
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    if (key)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return (*key)[a] < (*key)[b]; });
    else
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
    for (int i : order) per[owner[i]].push_back(i);
    out_items.clear();
    cta_ptr.assign(ncta + 1, 0);
    if (perm) perm->clear();
    for (int c = 0; c < ncta; ++c) {
        for (int i : per[c]) {
            out_items.push_back(items[i]);
            if (perm) perm->push_back(i);
        }
        cta_ptr[c + 1] = (int)out_items.size();
    }
}

// Load of one tensor-core tile in K stages: every stage moves the same bytes
// (A planes padded to 128 rows) and takes the same MMAs whatever the tile's
// real row count, so the rows do not enter; a tile also pays its accumulator
// drain, about two stages.  A pair of row tiles (the paired-tile kernels, 16
// K values per stage) costs twice the stages of its first tile.
static double tile_cost(int64_t K, int ks) { return (double)((K + ks - 1) / ks) + 2.0; }
static double pair_cost(double single32) { return 2.0 * (single32 - 2.0) + 2.0; }

// Z-order (Morton) code of every atom centre, from its x, y position in the
// array's bounding box quantised to 16 bits per axis
static std::vector<uint64_t> atom_zorder(const Op& op) {
    // (a joined operator of several problems keeps no centres: one key for all)
    if (op.centres.size() < 3 * (size_t)op.N) return std::vector<uint64_t>(op.N, 0);
    double lo[2] = {std::numeric_limits<double>::max(), std::numeric_limits<double>::max()};
    double hi[2] = {-lo[0], -lo[1]};
    for (int a = 0; a < op.N; ++a)
        for (int d = 0; d < 2; ++d) {
            lo[d] = std::min(lo[d], op.centres[3 * a + d]);
            hi[d] = std::max(hi[d], op.centres[3 * a + d]);
        }
    std::vector<uint64_t> z(op.N);
    for (int a = 0; a < op.N; ++a) {
        uint32_t q[2];
        for (int d = 0; d < 2; ++d) {
            const double span = hi[d] - lo[d];
            const double f = span > 0 ? (op.centres[3 * a + d] - lo[d]) / span : 0.0;
            q[d] = (uint32_t)std::min(65535.0, std::max(0.0, std::floor(f * 65535.0 + 0.5)));
        }
        uint64_t code = 0;
        for (int bit = 15; bit >= 0; --bit) code = (code << 2) | (((q[1] >> bit) & 1u) << 1) | ((q[0] >> bit) & 1u);
        z[a] = code;
    }
    return z;
}

void build_apply_lists(Op& op) {
    const int nb = (int)op.blocks.size();
    std::vector<FarBlockDev> hb(std::max(nb, 1));
    int64_t toff = 0;
    for (int i = 0; i < nb; ++i) {
        auto& b = op.blocks[i];
        b.t_off_vec = toff;
        toff += b.rank;
        const int prob = op.block_prob.empty() ? 0 : op.block_prob[i];
        hb[i] = FarBlockDev{b.m, b.n, b.rank, b.nt, b.ns, b.t_off, b.s_off, prob, (long long)b.q_off,
                            (long long)b.rh_off, (long long)b.t_off_vec};
    }
    op.t_total = toff;
    upload(op.d_blocks, hb);
    upload(op.d_block_atoms, op.block_atoms.empty() ? std::vector<int>{0} : op.block_atoms);
    op.n_cta = op.ctx->n_sm * 3;

    // phase 1
    std::vector<int4> it1;
    std::vector<double> w1;
    // one item = up to 32 rows of R_b (8 warps x 4 rows); smaller blocks keep
    // whole rows together so that every warp of the CTA has work
    for (int i = 0; i < nb; ++i) {
        const auto& b = op.blocks[i];
        if (b.rank == 0) continue;
        int rc = 32;
        for (int k0 = 0; k0 < b.rank; k0 += rc) {
            int k1 = std::min(b.rank, k0 + rc);
            it1.push_back(make_int4(i, k0, k1, op.block_prob.empty() ? 0 : op.block_prob[i]));
            w1.push_back((double)(k1 - k0) * b.n);
        }
    }
    std::vector<int4> p1;
    std::vector<int> c1;
    pack_lpt(it1, w1, op.n_cta, p1, c1);
    op.n_p1_items = (int)p1.size();
    upload(op.d_p1_items, p1.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : p1);
    upload(op.d_p1_cta, c1);
    // the same items on two CTAs per SM: the multi-RHS kernels hold two CTAs
    // per SM (their register use), and a third list entry per SM would run as
    // a second wave
    op.n_cta_m = op.ctx->n_sm * 2;
    {
        std::vector<int4> q;
        std::vector<int> c;
        pack_lpt(it1, w1, op.n_cta_m, q, c);
        upload(op.d_p1m_items, q.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : q);
        upload(op.d_p1m_cta, c);
    }

    // phase 2: per atom the (block, slot) entries, then row chunks
    std::vector<std::vector<int2>> ent(op.N);
    for (int i = 0; i < nb; ++i) {
        const auto& b = op.blocks[i];
        if (b.rank == 0) continue;
        for (int s = 0; s < b.nt; ++s) ent[op.block_atoms[b.t_off + s]].push_back(make_int2(i, s));
    }
    std::vector<int> csr(op.N + 1, 0);
    std::vector<int2> flat;
    std::vector<double> rsum(op.N, 0.0);
    for (int a = 0; a < op.N; ++a) {
        for (auto e : ent[a]) {
            flat.push_back(e);
            rsum[a] += op.blocks[e.x].rank;
        }
        csr[a + 1] = (int)flat.size();
    }
    std::vector<int4> it2;
    std::vector<double> w2;
    const int rows_per_item = 128;
    for (int a = 0; a < op.N; ++a)
        for (int p0 = 0; p0 < op.np; p0 += rows_per_item) {
            int p1e = std::min(op.np, p0 + rows_per_item);
            it2.push_back(make_int4(a, p0, p1e, op.atom_prob.empty() ? 0 : op.atom_prob[a]));
            w2.push_back((double)(p1e - p0) * (rsum[a] + 1.0));
        }
    std::vector<int4> p2;
    std::vector<int> c2;
    pack_lpt(it2, w2, op.n_cta, p2, c2);
    op.n_p2_items = (int)p2.size();
    upload(op.d_p2_items, p2);
    upload(op.d_p2_cta, c2);
    {
        std::vector<int4> q;
        std::vector<int> c;
        pack_lpt(it2, w2, op.n_cta_m, q, c);
        upload(op.d_p2m_items, q);
        upload(op.d_p2m_cta, c);
    }

    // tensor-core path: 64-row output tiles (rows of R_b, rows of an atom)
    op.n_cta_tc = op.ctx->n_sm * 4;
    std::vector<int4> t1, t2;
    std::vector<double> wt1, wt2;
    for (int i = 0; i < nb; ++i) {
        const auto& b = op.blocks[i];
        for (int k0 = 0; k0 < b.rank; k0 += 64) {
            t1.push_back(make_int4(i, k0, std::min(b.rank, k0 + 64), 0));
            wt1.push_back(64.0 * b.n);
        }
    }
    for (int a = 0; a < op.N; ++a)
        for (int p0 = 0; p0 < op.np; p0 += 64) {
            t2.push_back(make_int4(a, p0, std::min(op.np, p0 + 64), 0));
            wt2.push_back(64.0 * (rsum[a] + 1.0));
        }
    std::vector<int4> q1, q2;
    std::vector<int> e1, e2;
    pack_lpt(t1, wt1, op.n_cta_tc, q1, e1);
    pack_lpt(t2, wt2, op.n_cta_tc, q2, e2);
    op.n_t1_items = (int)q1.size();
    op.n_t2_items = (int)q2.size();
    upload(op.d_t1_items, q1.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : q1);
    upload(op.d_t1_cta, e1);
    upload(op.d_t2_items, q2);
    upload(op.d_t2_cta, e2);
    upload(op.d_p2_csr, csr);
    upload(op.d_p2_ent, flat.empty() ? std::vector<int2>{make_int2(0, 0)} : flat);
    op.umma_ready = false;

    // shared-factor path: classes of blocks with the same factor storage, in
    // groups of up to Op::kShareGroup members; phase 1 items of 32 rows of R,
    // phase 2 items of one target slot and 128 rows of it
    {
        std::map<std::pair<long long, int>, std::vector<int>> cls;
        std::vector<long long> poff(std::max(nb, 1), 0);
        int64_t ptot = 0;
        for (int i = 0; i < nb; ++i) {
            const auto& b = op.blocks[i];
            poff[i] = ptot;
            if (b.rank == 0) continue;
            ptot += (int64_t)b.nt * op.np;
            cls[{(long long)b.rh_off, op.block_prob.empty() ? 0 : op.block_prob[i]}].push_back(i);
        }
        std::vector<int> cmem;
        std::vector<int4> c1, c2;
        std::vector<double> v1, v2;
        int64_t nmem = 0;
        for (const auto& kv : cls) {
            const auto& mem = kv.second;
            nmem += (int64_t)mem.size();
            const auto& b = op.blocks[mem[0]];
            const size_t G = Op::kShareGroup;
            for (size_t g = 0; g < mem.size(); g += G) {
                const int first = (int)cmem.size();
                const int cnt = (int)std::min<size_t>(G, mem.size() - g);
                for (int j = 0; j < cnt; ++j) cmem.push_back(mem[g + j]);
                for (int k0 = 0; k0 < b.rank; k0 += 32) {
                    const int k1 = std::min(b.rank, k0 + 32);
                    c1.push_back(make_int4(first, k0, k1, cnt));
                    v1.push_back((double)(k1 - k0) * b.n * (1.0 + 0.25 * cnt));
                }
                for (int sl = 0; sl < b.nt; ++sl)
                    for (int p0 = 0; p0 < op.np; p0 += 128) {
                        const int p1e = std::min(op.np, p0 + 128);
                        c2.push_back(make_int4(first, sl, p0 | (p1e << 16), cnt));
                        v2.push_back((double)(p1e - p0) * b.rank * (1.0 + 0.25 * cnt));
                    }
            }
        }
        op.share_mean = cls.empty() ? 1.0 : (double)nmem / (double)cls.size();
        op.part_total = ptot;
        op.n_cta_c = op.ctx->n_sm * 3;
        std::vector<int4> q1, q2;
        std::vector<int> e1, e2;
        pack_lpt(c1, v1, op.n_cta_c, q1, e1);
        pack_lpt(c2, v2, op.n_cta_c, q2, e2);
        op.n_c1_items = (int)q1.size();
        op.n_c2_items = (int)q2.size();
        upload(op.d_c1_items, q1.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : q1);
        upload(op.d_c1_cta, e1);
        upload(op.d_c2_items, q2.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : q2);
        upload(op.d_c2_cta, e2);
        upload(op.d_cmem, cmem.empty() ? std::vector<int>{0} : cmem);
        upload(op.d_poff, poff);
        op.d_part.release();  // sized on first use (shared_reserve)
    }
}

void build_umma_lists(Op& op) {
    if (op.umma_ready) return;
    const int nb = (int)op.blocks.size();
    constexpr int kRows = 128;
    op.n_cta_u = op.ctx->n_sm * 2;
    // phase 1: blocks with the same source atoms share x_J, so their R rows
    // are stacked into one tall operand and cut into 128-row tiles
    std::map<std::vector<int>, std::vector<int>> groups;
    for (int i = 0; i < nb; ++i) {
        const auto& b = op.blocks[i];
        if (b.rank == 0) continue;
        std::vector<int> key(op.block_atoms.begin() + b.s_off, op.block_atoms.begin() + b.s_off + b.ns);
        groups[key].push_back(i);
    }
    const std::vector<uint64_t> zc = atom_zorder(op);
    std::vector<long long> rowoff;
    std::vector<int> rowt;
    std::vector<int4> it1;
    std::vector<double> w1;
    std::vector<uint64_t> key1, key2;  // spatial keys: the source atoms' lowest Z-order code, the atom's
    for (const auto& kv : groups) {
        const int rep = kv.second.front();
        uint64_t zmin = ~0ull;
        for (int a : kv.first) zmin = std::min(zmin, zc[a]);
        const int64_t start = (int64_t)rowoff.size();
        for (int i : kv.second) {
            const auto& b = op.blocks[i];
            for (int k = 0; k < b.rank; ++k) {
                rowoff.push_back((long long)(b.rh_off + (int64_t)k * b.n));
                rowt.push_back((int)(b.t_off_vec + k));
            }
        }
        const int64_t total = (int64_t)rowoff.size() - start;
        for (int64_t r0 = 0; r0 < total; r0 += kRows) {
            const int nr = (int)std::min<int64_t>(kRows, total - r0);
            it1.push_back(make_int4(rep, (int)(start + r0), nr, op.block_prob.empty() ? 0 : op.block_prob[rep]));
            w1.push_back(tile_cost(op.blocks[rep].n, 32));
            key1.push_back(zmin);
        }
    }
    // phase 2: per atom every (block, rank index) as one virtual K axis
    std::vector<std::vector<int2>> ent(op.N);
    for (int i = 0; i < nb; ++i) {
        const auto& b = op.blocks[i];
        if (b.rank == 0) continue;
        for (int s = 0; s < b.nt; ++s) ent[op.block_atoms[b.t_off + s]].push_back(make_int2(i, s));
    }
    std::vector<long long> qoff, kptr(op.N + 1, 0);
    std::vector<int> tidx;
    std::vector<int4> it2;
    std::vector<double> w2;
    for (int a = 0; a < op.N; ++a) {
        for (auto e : ent[a]) {
            const auto& b = op.blocks[e.x];
            for (int k = 0; k < b.rank; ++k) {
                qoff.push_back((long long)(b.q_off + (int64_t)e.y * op.np + (int64_t)k * b.m));
                tidx.push_back((int)(b.t_off_vec + k));
            }
        }
        kptr[a + 1] = (long long)qoff.size();
        const double K = (double)(kptr[a + 1] - kptr[a]);
        for (int p0 = 0; p0 < op.np; p0 += kRows) {
            const int p1 = std::min(op.np, p0 + kRows);
            it2.push_back(make_int4(a, p0, p1, op.atom_prob.empty() ? 0 : op.atom_prob[a]));
            w2.push_back(tile_cost((int64_t)K, 32));
            key2.push_back(zc[a]);
        }
    }
    std::vector<int4> q1, q2, r1, r2;
    std::vector<int> e1, e2, f1, f2, p1, p2, pr1, pr2;
    pack_lpt(it1, w1, op.n_cta_u, q1, e1, &p1, &key1);
    pack_lpt(it2, w2, op.n_cta_u, q2, e2, &p2, &key2);
    // the same items mapped to one CTA per SM (warp-specialised kernels)
    pack_lpt(it1, w1, op.ctx->n_sm, r1, f1, &pr1, &key1);
    pack_lpt(it2, w2, op.ctx->n_sm, r2, f2, &pr2, &key2);
    op.n_u1_items = (int)q1.size();
    op.n_u2_items = (int)q2.size();
    upload(op.d_u1_rowoff, rowoff.empty() ? std::vector<long long>{0} : rowoff);
    upload(op.d_u1_rowt, rowt.empty() ? std::vector<int>{0} : rowt);
    upload(op.d_u1_items, q1.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : q1);
    upload(op.d_u1_cta, e1);
    upload(op.d_u2_qoff, qoff.empty() ? std::vector<long long>{0} : qoff);
    upload(op.d_u2_tidx, tidx.empty() ? std::vector<int>{0} : tidx);
    upload(op.d_u2_kptr, kptr);
    upload(op.d_u2_items, q2.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : q2);
    upload(op.d_u2_cta, e2);
    // packed variant: every item's A operand as whole 32-wide K stages, item
    // after item in work-list order; offsets in stages
    auto stage_offsets = [](const std::vector<int4>& items, auto nk_of, std::vector<long long>& off) {
        off.assign(items.size() + 1, 0);
        for (size_t i = 0; i < items.size(); ++i) off[i + 1] = off[i] + (nk_of(items[i]) + 31) / 32;
    };
    std::vector<long long> pk1, pk2;
    stage_offsets(q1, [&](const int4& it) { return (long long)op.blocks[it.x].n; }, pk1);
    stage_offsets(q2, [&](const int4& it) { return kptr[it.x + 1] - kptr[it.x]; }, pk2);
    op.u1_stages = pk1.back();
    op.u2_stages = pk2.back();
    upload(op.d_u1_pk, pk1);
    upload(op.d_u2_pk, pk2);
    // stage offsets of the one-CTA-per-SM lists: the planes stay where the
    // first list put them (item i of that list at pk[i])
    auto remap = [](const std::vector<int>& perm_from, const std::vector<int>& perm_to,
                    const std::vector<long long>& pk) {
        std::vector<int> pos(perm_from.size());
        for (size_t i = 0; i < perm_from.size(); ++i) pos[perm_from[i]] = (int)i;
        std::vector<long long> out(perm_to.size() + 1, pk.back());
        for (size_t i = 0; i < perm_to.size(); ++i) out[i] = pk[pos[perm_to[i]]];
        return out;
    };
    upload(op.d_w1_items, r1.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : r1);
    upload(op.d_w1_cta, f1);
    upload(op.d_w1_pk, remap(p1, pr1, pk1));
    upload(op.d_w2_items, r2.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : r2);
    upload(op.d_w2_cta, f2);
    upload(op.d_w2_pk, remap(p2, pr2, pk2));
    // pairs of items with one B operand (the paired-tile kernels): two
    // consecutive row tiles of one source group (phase 1) or of one target
    // atom (phase 2); a leftover tile goes alone, its second item with 0 rows
    auto pair_lists = [&](const std::vector<int4>& items, const std::vector<double>& w,
                          const std::vector<uint64_t>& key, const std::vector<int>& perm_from,
                          const std::vector<long long>& pk, auto same_b, auto empty_of, DevBuf& d_items,
                          DevBuf& d_items_b, DevBuf& d_cta, DevBuf& d_pk, DevBuf& d_pk_b) {
        std::vector<int> pos(perm_from.size());
        for (size_t i = 0; i < perm_from.size(); ++i) pos[perm_from[i]] = (int)i;
        std::vector<int2> pairs;
        std::vector<int4> first;
        std::vector<double> pw;
        std::vector<uint64_t> pkey;
        for (size_t i = 0; i < items.size(); ++i) {
            const bool two = i + 1 < items.size() && same_b(items[i], items[i + 1]);
            pairs.push_back(make_int2((int)i, two ? (int)i + 1 : -1));
            first.push_back(items[i]);
            pw.push_back(pair_cost(w[i]));
            pkey.push_back(key[i]);
            if (two) ++i;
        }
        std::vector<int4> out;
        std::vector<int> cta, perm;
        pack_lpt(first, pw, op.ctx->n_sm, out, cta, &perm, &pkey);
        std::vector<int4> ib(out.size());
        std::vector<long long> pa(out.size() + 1, pk.back()), pb(out.size() + 1, 0);
        for (size_t k = 0; k < out.size(); ++k) {
            const int2 pr = pairs[perm[k]];
            pa[k] = pk[pos[pr.x]];
            ib[k] = pr.y >= 0 ? items[pr.y] : empty_of(items[pr.x]);
            pb[k] = pr.y >= 0 ? pk[pos[pr.y]] : 0;
        }
        upload(d_items, out.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : out);
        upload(d_items_b, ib.empty() ? std::vector<int4>{make_int4(0, 0, 0, 0)} : ib);
        upload(d_cta, cta);
        upload(d_pk, pa);
        upload(d_pk_b, pb);
    };
    // phase 1 items (rep block, first row, rows, problem); phase 2 (atom, p0, p1, problem)
    pair_lists(
        it1, w1, key1, p1, pk1,
        [](const int4& a, const int4& b) { return a.x == b.x && b.y == a.y + a.z; },
        [](const int4& a) { return make_int4(a.x, a.y, 0, a.w); }, op.d_x1_items, op.d_x1_items_b, op.d_x1_cta,
        op.d_x1_pk, op.d_x1_pk_b);
    pair_lists(
        it2, w2, key2, p2, pk2, [](const int4& a, const int4& b) { return a.x == b.x && b.y == a.z; },
        [](const int4& a) { return make_int4(a.x, 0, 0, a.w); }, op.d_x2_items, op.d_x2_items_b, op.d_x2_cta,
        op.d_x2_pk, op.d_x2_pk_b);
    op.umma_packed = false;
    op.umma_pack_failed = false;
    op.d_u1_pack.release();
    op.d_u2_pack.release();
    op.umma_ready = true;
}

}  // namespace vie
