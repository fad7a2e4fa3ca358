// Host-side construction of the surface codes' Tanner graphs (no GPU calls).
//
// The codes are the hypergraph products (HGP) of repetition codes described
// in Sec. II-A and Sec. IV-B of the paper: the toric code [[2L^2,2,L]] from
// the cyclic [L,1] repetition code, the planar code [[2L^2-2L+1,1,L]] from
// the open one, and the XZZX code as the planar code with a Hadamard on every
// qubit of the second HGP block.  They are laid out here directly on the
// lattice: block 1 is an L x L grid of qubits (a, b), block 2 a grid of
// qubits (r, s) on the faces; an X-type check (r, b) touches block-1 qubits
// (r, b), (r+1, b) and block-2 qubits (r, b-1), (r, b); a Z-type check (a, s)
// touches block-1 qubits (a, s), (a, s+1) and block-2 qubits (a-1, s), (a, s)
// (indices wrap around on the torus and are dropped outside the grid on the
// plane).  Qubit order: block 1 row-major, then block 2 row-major; check
// order: X-type rows, then Z-type rows.
#include <algorithm>
#include <array>
#include <cstring>
#include <new>

#include "bpq_internal.h"

namespace bpq {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

int finish_csr(bpq_tanner *t, std::vector<std::vector<std::pair<int, uint8_t>>> &rows) {
    t->M = (int)rows.size();
    t->chk_ptr.assign(t->M + 1, 0);
    t->chk_var.clear();
    t->chk_pauli.clear();
    for (int i = 0; i < t->M; ++i) {
        auto &r = rows[i];
        std::sort(r.begin(), r.end());
        for (size_t n = 1; n < r.size(); ++n)
            if (r[n].first == r[n - 1].first) return fail(BPQ_EINVAL, "duplicate qubit in a check");
        t->chk_ptr[i] = (int)t->chk_var.size();
        for (auto &e : r) {
            t->chk_var.push_back(e.first);
            t->chk_pauli.push_back(e.second);
        }
    }
    t->chk_ptr[t->M] = (int)t->chk_var.size();
    t->E = (int)t->chk_var.size();
    return build_tables(t);
}

int build_tables(bpq_tanner *t) {
    const int N = t->N, M = t->M;
    if (N < 1 || M < 0) return fail(BPQ_EINVAL, "empty code");
    if (std::max(N, M) > kMaxNodes) return fail(BPQ_EINVAL, "code larger than the decoder's node limit");
    if (4 * (long)N >= kNoSlot) return fail(BPQ_EINVAL, "too many qubits for 16-bit slots");
    // per-qubit edge lists in increasing check order
    std::vector<std::vector<int>> var_edges(N);
    for (int i = 0; i < M; ++i) {
        int deg = t->chk_ptr[i + 1] - t->chk_ptr[i];
        if (deg > kMaxDeg) return fail(BPQ_EINVAL, "check degree above 4");
        for (int e = t->chk_ptr[i]; e < t->chk_ptr[i + 1]; ++e) var_edges[t->chk_var[e]].push_back(e);
    }
    for (int j = 0; j < N; ++j)
        if ((int)var_edges[j].size() > kMaxDeg) return fail(BPQ_EINVAL, "qubit degree above 4");

    const int M_pad = (M + 15) & ~15, N_pad = (N + 15) & ~15;
    const size_t bytes = (size_t)M_pad * 8 + M_pad + N_pad;
    t->table.assign((bytes + 15) & ~size_t(15), 0);
    t->off_chk_pauli = (uint32_t)(M_pad * 8);
    t->off_var_pauli = (uint32_t)(M_pad * 8 + M_pad);
    uint16_t *slot = reinterpret_cast<uint16_t *>(t->table.data());
    uint8_t *cp = t->table.data() + t->off_chk_pauli;
    uint8_t *vp = t->table.data() + t->off_var_pauli;
    for (int k = 0; k < M_pad * 4; ++k) slot[k] = kNoSlot;
    t->var_canon.assign((size_t)4 * N, -1);

    // Qubit j's edges occupy slots 4j .. 4j+3, its k-th edge at position
    // (k + (j >> 3)) mod 4.  The rotation spreads the check pass's accesses
    // (32 consecutive checks touch about 32 consecutive qubits) over all 32
    // shared-memory banks instead of the 8 that slot 4j + k would hit.
    std::vector<int> slot_of_edge(t->E, -1);
    for (int j = 0; j < N; ++j) {
        uint8_t bits = 0;
        for (size_t k = 0; k < var_edges[j].size(); ++k) {
            const int e = var_edges[j][k];
            const int pos = ((int)k + (j >> 3)) & 3;
            slot_of_edge[e] = 4 * j + pos;
            t->var_canon[4 * j + pos] = e;
            bits |= (uint8_t)(t->chk_pauli[e] << (2 * pos));
        }
        vp[j] = bits;
    }
    for (int i = 0; i < M; ++i) {
        uint8_t bits = 0;
        for (int e = t->chk_ptr[i], n = 0; e < t->chk_ptr[i + 1]; ++e, ++n) {
            slot[4 * i + n] = (uint16_t)slot_of_edge[e];
            bits |= (uint8_t)(t->chk_pauli[e] << (2 * n));
        }
        cp[i] = bits;
    }

    // split layout (see bpq_tanner::split)
    t->split = true;
    for (int j = 0; j < N && t->split; ++j) {
        int nx = 0, nz = 0;
        for (int e : var_edges[j]) {
            const uint8_t p = t->chk_pauli[e];
            nx += p == 1;
            nz += p == 3;
            if (p == 2) t->split = false;
        }
        if (nx > 2 || nz > 2) t->split = false;
    }
    t->full = t->split;
    for (int i = 0; i < M && t->full; ++i) t->full = t->chk_ptr[i + 1] - t->chk_ptr[i] == 4;
    for (int j = 0; j < N && t->full; ++j) {
        int nx = 0, nz = 0;
        for (int e : var_edges[j]) {
            nx += t->chk_pauli[e] == 1;
            nz += t->chk_pauli[e] == 3;
        }
        t->full = nx == 2 && nz == 2;
    }
    t->table_split.clear();
    t->var_canon_split.clear();
    if (t->split) {
        const int n4 = (N + 3) & ~3;
        t->table_split.assign(t->table.size(), 0);
        t->var_canon_split.assign((size_t)4 * n4, -1);
        uint16_t *slot2 = reinterpret_cast<uint16_t *>(t->table_split.data());
        uint8_t *cp2 = t->table_split.data() + t->off_chk_pauli;
        uint8_t *vp2 = t->table_split.data() + t->off_var_pauli;
        for (int k = 0; k < M_pad * 4; ++k) slot2[k] = kNoSlot;
        for (int j = 0; j < N; ++j) {
            int nx = 0, nz = 0;
            uint8_t bits = 0;
            for (int e : var_edges[j]) {
                const uint8_t p = t->chk_pauli[e];
                const int pos = p == 1 ? nx++ : 2 + nz++;
                slot_of_edge[e] = pos * n4 + j;
                t->var_canon_split[(size_t)pos * n4 + j] = e;
                bits |= (uint8_t)(p << (2 * pos));
            }
            vp2[j] = bits;
        }
        for (int i = 0; i < M; ++i)
            for (int e = t->chk_ptr[i], n = 0; e < t->chk_ptr[i + 1]; ++e, ++n)
                slot2[4 * i + n] = (uint16_t)slot_of_edge[e];
        std::memcpy(cp2, cp, (size_t)M_pad);
    }
    return build_serial_table(t);
}

namespace {
// Message slots of the serial kernels' edges: slot = bank + 32 * row, with
// bank chosen greedily so that the edges one warp instruction touches (the
// k-th edge, or its check's r-th other edge, of the qubits of one 32-lane
// step of a level) fall in distinct banks where possible: distinct slots
// mod 32 across the warp (32-bit accesses of the one-shot kernel) and
// distinct slots mod 16 within each half-warp (the 64-bit slot accesses of
// the two-shot kernel are served half a warp at a time).  Edges are
// coloured in sweep order; each bank holds at most ceil(E / 32) + 1 edges.
std::vector<int> colour_serial_slots(const std::vector<std::array<int, 4>> &at, const std::vector<int> &edge_chk,
                                     const std::vector<int32_t> &chk_ptr, const std::vector<int> &order,
                                     const std::vector<int> &lp, int E, int *nslots) {
    const int nlev = (int)lp.size() - 1;
    struct Use {
        int edge, lane;
    };
    std::vector<std::vector<Use>> groups;
    for (int l = 0; l < nlev; ++l)
        for (int s0 = lp[l]; s0 < lp[l + 1]; s0 += 32) {
            const int s1 = std::min(lp[l + 1], s0 + 32);
            for (int k = 0; k < 4; ++k)
                for (int r = 0; r < 4; ++r) {
                    std::vector<Use> g;
                    for (int v = s0; v < s1; ++v) {
                        const int e = at[order[v]][k];
                        if (e < 0) continue;
                        const int i = edge_chk[e];
                        if (r == 3) {
                            g.push_back({e, v - s0});
                            continue;
                        }
                        int f = 0;
                        for (int x = chk_ptr[i]; x < chk_ptr[i + 1]; ++x)
                            if (x != e && f++ == r) g.push_back({x, v - s0});
                    }
                    if (!g.empty()) groups.push_back(std::move(g));
                }
        }
    struct Member {
        int group, lane;
    };
    std::vector<std::vector<Member>> edge_groups(E);  // the groups of an edge, with its lane in each
    for (int gi = 0; gi < (int)groups.size(); ++gi)
        for (const Use &u : groups[gi]) edge_groups[u.edge].push_back({gi, u.lane});
    const int cap = (E + 31) / 32 + 1;
    std::vector<int> bank(E, -1), fill(32, 0), slot(E);
    for (int v = 0; v < (int)order.size(); ++v)
        for (int e : at[order[v]]) {
            if (e < 0) continue;
            int cost[32] = {0};
            for (const Member &eg : edge_groups[e])
                for (const Use &u : groups[eg.group]) {
                    const int b = bank[u.edge];
                    if (b < 0) continue;
                    ++cost[b];
                    if ((u.lane < 16) == (eg.lane < 16)) {
                        ++cost[b & 15];
                        ++cost[(b & 15) + 16];
                    }
                }
            int best = -1;
            for (int b = 0; b < 32; ++b)
                if (fill[b] < cap && (best < 0 || cost[b] < cost[best] || (cost[b] == cost[best] && fill[b] < fill[best])))
                    best = b;
            bank[e] = best;
            slot[e] = best + 32 * fill[best]++;
        }
    int top = 0;
    for (int b = 0; b < 32; ++b) top = std::max(top, fill[b]);
    *nslots = 32 * top;
    return slot;
}
}  // namespace

int build_serial_table(bpq_tanner *t) {
    const int N = t->N, M = t->M, E = t->E;
    // level(j) = 1 + the largest level among the earlier qubits sharing a check with j
    std::vector<std::vector<int>> var_edges(N);
    std::vector<int> edge_chk(E);
    for (int i = 0; i < M; ++i)
        for (int e = t->chk_ptr[i]; e < t->chk_ptr[i + 1]; ++e) {
            var_edges[t->chk_var[e]].push_back(e);
            edge_chk[e] = i;
        }
    std::vector<int> level(N), chk_last(M, -1), chk_lastq(M, -1);
    int nlevels = 0;
    for (int j = 0; j < N; ++j) {
        int l = 0;
        for (int e : var_edges[j]) l = std::max(l, chk_last[edge_chk[e]] + 1);
        level[j] = l;
        for (int e : var_edges[j]) {
            chk_last[edge_chk[e]] = l;
            chk_lastq[edge_chk[e]] = j;  // qubits in index order: the last one stays
        }
        nlevels = std::max(nlevels, l + 1);
    }
    std::vector<int> order(N);
    for (int j = 0; j < N; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return level[x] < level[y]; });
    std::vector<int> lp(nlevels + 1);
    for (int l = 0, v = 0; l <= nlevels; ++l) {
        while (v < N && level[order[v]] < l) ++v;
        lp[l] = v;
    }
    // edge at each of a qubit's four positions (-1: padding): in increasing
    // check order, or (split layout) the X edges at 0, 1 and the Z edges at
    // 2, 3
    std::vector<std::array<int, 4>> at(N);
    for (int j = 0; j < N; ++j) {
        at[j] = {-1, -1, -1, -1};
        int nx = 0, nz = 0;
        for (int q = 0; q < (int)var_edges[j].size(); ++q) {
            const int e = var_edges[j][q];
            at[j][!t->split ? q : t->chk_pauli[e] == 1 ? nx++ : 2 + nz++] = e;
        }
    }
    int nslots = 0;
    const std::vector<int> slot = colour_serial_slots(at, edge_chk, t->chk_ptr, order, lp, E, &nslots);
    if (nslots + 2 > 0xFFFF || M >= 0xFFFF || E >= 0xFFFF || N > 0xFFFF)
        return fail(BPQ_EINVAL, "code too large for the serial table");
    const uint16_t kZero = (uint16_t)nslots, kTrash = (uint16_t)(nslots + 1);

    const size_t vars_bytes = sizeof(SerialVar) * (size_t)N;
    const size_t off_levels = vars_bytes;
    const size_t off_canon = (off_levels + 2 * (size_t)(nlevels + 1) + 15) & ~size_t(15);
    const size_t bytes = (off_canon + 8 * (size_t)N + 15) & ~size_t(15);
    t->serial.assign(bytes, 0);
    SerialVar *vars = reinterpret_cast<SerialVar *>(t->serial.data());
    uint16_t *lpt = reinterpret_cast<uint16_t *>(t->serial.data() + off_levels);
    uint16_t *canon = reinterpret_cast<uint16_t *>(t->serial.data() + off_canon);
    for (int v = 0; v < N; ++v) {
        const int j = order[v];
        SerialVar &sv = vars[v];
        sv.j = (uint16_t)j;
        sv.pauli = 0;
        sv.last = 0;
        sv.real = 0;
        for (int k = 0; k < 4; ++k) {
            sv.own[k] = kTrash;
            sv.chk[k] = 0;
            canon[4 * v + k] = (uint16_t)E;
            for (int f = 0; f < 3; ++f) sv.oth[k][f] = kZero;
        }
        for (int k = 0; k < 4; ++k) {
            const int e = at[j][k];
            if (e < 0) continue;
            const int i = edge_chk[e];
            sv.real |= (uint8_t)(1u << k);
            sv.own[k] = (uint16_t)slot[e];
            sv.chk[k] = (uint16_t)i;
            canon[4 * v + k] = (uint16_t)e;
            sv.pauli |= (uint8_t)(t->chk_pauli[e] << (2 * k));
            if (chk_lastq[i] == j) sv.last |= (uint8_t)(1u << k);
            int f = 0;
            for (int x = t->chk_ptr[i]; x < t->chk_ptr[i + 1]; ++x)
                if (x != e) sv.oth[k][f++] = (uint16_t)slot[x];
        }
    }
    for (int l = 0; l <= nlevels; ++l) lpt[l] = (uint16_t)lp[l];
    t->serial_levels = nlevels;
    t->serial_slots = nslots;
    t->serial_off_levels = (uint32_t)off_levels;
    t->serial_off_canon = (uint32_t)off_canon;
    return BPQ_OK;
}

}  // namespace bpq

using bpq::fail;

namespace {

constexpr uint8_t PX = 1, PZ = 3;

int build_surface(int code, int L, bpq_tanner *t) {
    const bool torus = code == BPQ_TORIC;
    const int n1 = L;                    // block-1 grid is L x L
    const int m1 = torus ? L : L - 1;    // block-2 grid is m1 x m1
    t->N = n1 * n1 + m1 * m1;
    t->K = torus ? 2 : 1;
    auto q1 = [&](int a, int b) { return a * n1 + b; };
    auto q2 = [&](int r, int s) { return n1 * n1 + r * m1 + s; };
    auto wrap = [&](int x, int n) { return torus ? (x % n + n) % n : x; };
    const bool xzzx = code == BPQ_XZZX;
    const uint8_t b2x = xzzx ? PZ : PX, b2z = xzzx ? PX : PZ;  // Hadamard on block 2

    std::vector<std::vector<std::pair<int, uint8_t>>> rows;
    // X-type checks (r, b): r in [m1], b in [n1]
    for (int r = 0; r < m1; ++r)
        for (int b = 0; b < n1; ++b) {
            std::vector<std::pair<int, uint8_t>> row;
            row.push_back({q1(r, b), PX});
            row.push_back({q1(wrap(r + 1, n1), b), PX});
            for (int s : {b - 1, b}) {
                int sw = wrap(s, m1);
                if (sw >= 0 && sw < m1) row.push_back({q2(r, sw), b2x});
            }
            rows.push_back(row);
        }
    // Z-type checks (a, s): a in [n1], s in [m1]
    for (int a = 0; a < n1; ++a)
        for (int s = 0; s < m1; ++s) {
            std::vector<std::pair<int, uint8_t>> row;
            row.push_back({q1(a, s), PZ});
            row.push_back({q1(a, wrap(s + 1, n1)), PZ});
            for (int r : {a - 1, a}) {
                int rw = wrap(r, m1);
                if (rw >= 0 && rw < m1) row.push_back({q2(rw, s), b2z});
            }
            rows.push_back(row);
        }
    // Logical operators in closed form: X on block-1 row 0 and Z on block-1
    // column 0 (both commute with every check and overlap on one qubit); on
    // the torus also X on block-2 column 0 and Z on block-2 row 0.
    t->logicals.assign((size_t)2 * t->K * t->N, 0);
    for (int b = 0; b < n1; ++b) t->logicals[0 * t->N + q1(0, b)] = PX;
    for (int a = 0; a < n1; ++a) t->logicals[1 * t->N + q1(a, 0)] = PZ;
    if (torus) {
        for (int r = 0; r < m1; ++r) t->logicals[2 * t->N + q2(r, 0)] = PX;
        for (int s = 0; s < m1; ++s) t->logicals[3 * t->N + q2(0, s)] = PZ;
    }
    t->code = code;
    t->d = L;
    return bpq::finish_csr(t, rows);
}

}  // namespace

extern "C" {

void bpq_default_params(int variant, bpq_params *out) {
    if (!out) return;
    out->alpha = variant == BPQ_ADAGRAD ? 5.0f : (variant == BPQ_PLAIN || variant == BPQ_AEWA) ? 1.0f : 0.5f;
    out->gamma = 0.0f;
    out->eps = 1e-8f;
    out->msg_clip = 30.0f;
    out->adagrad_g_from_iter1 = 1;
}

int bpq_build_tanner(int code, int d, bpq_tanner **out) {
    if (!out) return fail(BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (code != BPQ_PLANAR && code != BPQ_TORIC && code != BPQ_XZZX)
        return fail(BPQ_EINVAL, "unknown code kind");
    if (d < (code == BPQ_TORIC ? 3 : 2) || d > 32) return fail(BPQ_EINVAL, "distance out of range");
    bpq_tanner *t = new (std::nothrow) bpq_tanner();
    if (!t) return fail(BPQ_ENOMEM, "allocation failed");
    int rc = build_surface(code, d, t);
    if (rc) { delete t; return rc; }
    *out = t;
    return BPQ_OK;
}

int bpq_tanner_from_paulis(int M, int N, const uint8_t *H, bpq_tanner **out) {
    if (!out) return fail(BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 0 || N < 1 || (M > 0 && !H)) return fail(BPQ_EINVAL, "bad sizes or NULL matrix");
    if (std::max(N, M) > bpq::kMaxNodes) return fail(BPQ_EINVAL, "matrix too large");
    bpq_tanner *t = new (std::nothrow) bpq_tanner();
    if (!t) return fail(BPQ_ENOMEM, "allocation failed");
    t->N = N;
    std::vector<std::vector<std::pair<int, uint8_t>>> rows(M);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < N; ++j) {
            uint8_t p = H[(size_t)i * N + j];
            if (p > 3) { delete t; return fail(BPQ_EINVAL, "Pauli code above 3"); }
            if (p) rows[i].push_back({j, p});
        }
    int rc = bpq::finish_csr(t, rows);
    if (rc) { delete t; return rc; }
    *out = t;
    return BPQ_OK;
}

int bpq_tanner_set_logicals(bpq_tanner *t, int n_logicals, const uint8_t *L) {
    if (!t || n_logicals < 0 || (n_logicals % 2) || (n_logicals && !L))
        return fail(BPQ_EINVAL, "bad logical operators");
    if (t->dev_blob) return fail(BPQ_ESTATE, "tanner already uploaded");
    for (size_t k = 0; k < (size_t)n_logicals * t->N; ++k)
        if (L[k] > 3) return fail(BPQ_EINVAL, "Pauli code above 3");
    t->logicals.assign(L, L + (size_t)n_logicals * t->N);
    t->K = n_logicals / 2;
    return BPQ_OK;
}

int bpq_tanner_info(const bpq_tanner *t, int *N, int *M, int *E, int *K) {
    if (!t) return fail(BPQ_EINVAL, "tanner is NULL");
    if (N) *N = t->N;
    if (M) *M = t->M;
    if (E) *E = t->E;
    if (K) *K = t->K;
    return BPQ_OK;
}

int bpq_tanner_layout(const bpq_tanner *t, int *layout) {
    if (!t || !layout) return fail(BPQ_EINVAL, "NULL argument");
    *layout = t->full ? 2 : t->split ? 1 : 0;
    return BPQ_OK;
}

int bpq_tanner_export(const bpq_tanner *t, int32_t *chk_ptr, int32_t *chk_var, uint8_t *pauli) {
    if (!t) return fail(BPQ_EINVAL, "tanner is NULL");
    if (chk_ptr) std::memcpy(chk_ptr, t->chk_ptr.data(), sizeof(int32_t) * (t->M + 1));
    if (chk_var) std::memcpy(chk_var, t->chk_var.data(), sizeof(int32_t) * t->E);
    if (pauli) std::memcpy(pauli, t->chk_pauli.data(), t->E);
    return BPQ_OK;
}

int bpq_tanner_logicals(const bpq_tanner *t, uint8_t *L) {
    if (!t || !L) return fail(BPQ_EINVAL, "NULL argument");
    if (t->logicals.empty()) return fail(BPQ_ESTATE, "no logical operators known");
    std::memcpy(L, t->logicals.data(), t->logicals.size());
    return BPQ_OK;
}

int bpq_version(void) { return 100; }

const char *bpq_last_error(void) { return bpq::g_last_error.c_str(); }

}  // extern "C"
