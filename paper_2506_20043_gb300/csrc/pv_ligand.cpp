// pv_ligand.cpp -- host construction of a ligand's device record: XS typing, rigid fragments
// and torsion tree (the POT parametrisation of Eq. 1), intra-ligand pair list (Eq. 3's
// e_intra) and its schedule into conflict-free rounds of 32 pairs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "pv_ligand.h"
#include "pv_terms.h"

namespace pv {

static int xs_type(int el, int don, int acc, bool c_polar) {
    if (el == 0) return c_polar ? 1 : 0;
    if (el == 1) return 2 + (don ? 1 : 0) + (acc ? 2 : 0);
    if (el == 2) return 6 + (don ? 1 : 0) + (acc ? 2 : 0);
    return 10;
}
static bool is_hyd(int t) { return t == 0; }
static bool is_don(int t) { return t == 3 || t == 5 || t == 7 || t == 9; }
static bool is_acc(int t) { return t == 4 || t == 5 || t == 8 || t == 9; }

// Orients every pair so that, per atom, sources and targets split its pairs evenly (an Euler
// circuit of the pair graph, with a dummy vertex joined to the odd-degree atoms, enters and
// leaves each atom equally often), then flips single pairs while that lowers the larger of a
// lane's source load and its target load (atoms l and l + lanes share lane l).
static void orient_pairs(int n, std::vector<std::pair<int, int>>& edges, int lanes) {
    const int m = (int)edges.size();
    if (m == 0) return;
    std::vector<std::pair<int, int>> E(edges);
    std::vector<int> deg(n + 1, 0);
    for (auto& e : E) { deg[e.first]++; deg[e.second]++; }
    for (int v = 0; v < n; ++v)
        if (deg[v] & 1) E.push_back({v, n});
    std::vector<std::vector<std::pair<int, int>>> adj(n + 1);
    for (int k = 0; k < (int)E.size(); ++k) {
        adj[E[k].first].push_back({E[k].second, k});
        adj[E[k].second].push_back({E[k].first, k});
    }
    std::vector<char> used(E.size(), 0);
    std::vector<size_t> ptr(n + 1, 0);
    for (int s0 = 0; s0 <= n; ++s0) {
        std::vector<std::pair<int, int>> stack{{s0, -1}};
        while (!stack.empty()) {
            const int v = stack.back().first;
            while (ptr[v] < adj[v].size() && used[adj[v][ptr[v]].second]) ++ptr[v];
            if (ptr[v] == adj[v].size()) {
                const int ein = stack.back().second;
                stack.pop_back();
                if (ein >= 0 && ein < m) edges[ein] = {stack.back().first, v};
            } else {
                const auto nx = adj[v][ptr[v]];
                used[nx.second] = 1;
                stack.push_back({nx.first, nx.second});
            }
        }
    }
    const int lm = lanes - 1;
    std::vector<int> load(lanes, 0), ind(lanes, 0);   // per lane: pairs as source, as target
    for (auto& e : edges) { load[e.first & lm]++; ind[e.second & lm]++; }
    for (bool changed = true; changed;) {
        changed = false;
        for (auto& e : edges) {
            const int s = e.first, t = e.second, ls = s & lm, lt = t & lm;
            if (ls == lt) continue;
            const int before = std::max(std::max(load[ls], load[lt]), std::max(ind[ls], ind[lt]));
            const int after = std::max(std::max(load[ls] - 1, load[lt] + 1), std::max(ind[ls] + 1, ind[lt] - 1));
            if (after < before || (after == before && load[lt] + 1 < load[ls] && ind[ls] + 1 < ind[lt])) {
                load[ls]--; load[lt]++; ind[ls]++; ind[lt]--;
                e = {t, s};
                changed = true;
            }
        }
    }
}

// Edge colouring of the bipartite multigraph source lanes x target lanes with as many colours
// (rounds) as its largest degree (Koenig): a pair gets a colour free at both ends, else the
// alternating path of the two candidate colours from its target lane is swapped first. In a round
// every lane then sends at most one pair and receives at most one.
static int colour_rounds(const std::vector<std::pair<int, int>>& edges, std::vector<int>& col, int lanes) {
    const int m = (int)edges.size();
    const int lm = lanes - 1;
    col.assign(m, -1);
    if (m == 0) return 0;
    std::vector<int> dl(lanes, 0), dr(lanes, 0);
    for (auto& e : edges) { dl[e.first & lm]++; dr[e.second & lm]++; }
    const int D = std::max(*std::max_element(dl.begin(), dl.end()), *std::max_element(dr.begin(), dr.end()));
    std::vector<int> Lc(lanes * D, -1), Rc(lanes * D, -1);   // edge holding colour c at a source / target lane
    for (int e = 0; e < m; ++e) {
        const int u = edges[e].first & lm, v = edges[e].second & lm;
        int a = 0, b = 0;
        while (Lc[u * D + a] >= 0) ++a;
        while (Rc[v * D + b] >= 0) ++b;
        if (Rc[v * D + a] >= 0) {
            std::vector<int> path;
            int x = v, c = a;
            bool right = true;
            for (;;) {
                const int f = right ? Rc[x * D + c] : Lc[x * D + c];
                if (f < 0) break;
                path.push_back(f);
                x = right ? (edges[f].first & lm) : (edges[f].second & lm);
                right = !right;
                c = c == a ? b : a;
            }
            for (int f : path) {
                Lc[(edges[f].first & lm) * D + col[f]] = -1;
                Rc[(edges[f].second & lm) * D + col[f]] = -1;
            }
            for (int f : path) {
                col[f] = col[f] == a ? b : a;
                Lc[(edges[f].first & lm) * D + col[f]] = f;
                Rc[(edges[f].second & lm) * D + col[f]] = f;
            }
        }
        col[e] = a;
        Lc[u * D + a] = e;
        Rc[v * D + a] = e;
    }
    return D;
}

// Shared-memory banks of the partner gathers. A quarter-warp (8 lanes) reads its partners' float4
// positions in one shared-memory wavefront when their atom indices differ modulo 8 (the 16-byte
// bank groups); partners of equal residue are read one after another. So a round costs, per
// quarter-warp, the largest number of its partners sharing a residue (empty slots read a dummy atom
// of a free residue), and a quarter-warp's rounds cost at least its largest count of pairs to one
// residue. Starting from the colouring above, a tabu search moves single pairs between rounds (the
// best of the moves of a random sample of the pairs in conflict), allowing a lane two pairs in a
// round for a while at a penalty, and keeps the best colouring without such a clash; it stops at
// that lower bound or after a fixed amount of work.
static void balance_banks(const std::vector<std::pair<int, int>>& edges, std::vector<int>& col, int D, int lanes) {
    const int m = (int)edges.size(), lm = lanes - 1, nq = lanes / 8;
    if (m == 0 || D < 2) return;
    auto src = [&](int e) { return edges[e].first & lm; };
    auto tgt = [&](int e) { return edges[e].second & lm; };
    auto cell = [&](int e, int c) { return (c * nq + (src(e) >> 3)) * 8 + (edges[e].second & 7); };
    std::vector<int> cnt((size_t)D * nq * 8, 0), S((size_t)lanes * D, 0), R((size_t)lanes * D, 0);
    for (int e = 0; e < m; ++e) {
        cnt[cell(e, col[e])]++;
        S[src(e) * D + col[e]]++;
        R[tgt(e) * D + col[e]]++;
    }
    auto cost = [&](int rq) {
        int c = 1;
        for (int k = 0; k < 8; ++k) c = std::max(c, cnt[rq * 8 + k]);
        return c;
    };
    std::vector<int> load(nq * 8, 0);
    for (int e = 0; e < m; ++e) load[(src(e) >> 3) * 8 + (edges[e].second & 7)]++;
    int bound = 0, soft = 0;
    for (int q = 0; q < nq; ++q) bound += std::max(D, *std::max_element(&load[q * 8], &load[q * 8] + 8));
    for (int rq = 0; rq < D * nq; ++rq) soft += cost(rq);
    int best = soft, clashes = 0;
    std::vector<int> best_col(col), tabu_until((size_t)m * D, 0);
    const int kPenalty = 3;                  // a lane's second pair in a round, in wavefronts
    const long long kWork = 2000000;         // pairs scanned and moves evaluated, at most
    const int kCand = 24;
    uint64_t rng = 0x9e3779b97f4a7c15ull;    // xorshift64, fixed seed: the schedule is reproducible
    auto next = [&]() { rng ^= rng << 13; rng ^= rng >> 7; rng ^= rng << 17; return rng; };
    long long work = 0;
    std::vector<int> cand;
    for (int it = 1; best > bound && work < kWork; ++it) {
        // the moves of up to kCand pairs, drawn from those in a clash or sharing a bank group
        cand.clear();
        for (int e = 0; e < m; ++e)
            if (S[src(e) * D + col[e]] > 1 || R[tgt(e) * D + col[e]] > 1 || cnt[cell(e, col[e])] > 1) cand.push_back(e);
        for (int i = 0; i < (int)cand.size() && i < kCand; ++i)
            std::swap(cand[i], cand[i + (int)(next() % (uint64_t)(cand.size() - i))]);
        if ((int)cand.size() > kCand) cand.resize(kCand);
        work += m + (long long)cand.size() * (D - 1);
        int best_d = 1 << 30, be = -1, bc = -1, ties = 0;
        for (int e : cand) {
            const int a = col[e], u = src(e), v = tgt(e), rqa = a * nq + (u >> 3);
            const int ca0 = cost(rqa);
            cnt[cell(e, a)]--;
            const int ca1 = cost(rqa);
            cnt[cell(e, a)]++;
            const int leave = (S[u * D + a] > 1 ? -1 : 0) + (R[v * D + a] > 1 ? -1 : 0);
            for (int b = 0; b < D; ++b) {
                if (b == a) continue;
                const int dc = leave + (S[u * D + b] > 0 ? 1 : 0) + (R[v * D + b] > 0 ? 1 : 0);
                const int rqb = b * nq + (u >> 3);
                const int cb0 = cost(rqb);
                cnt[cell(e, b)]++;
                const int cb1 = cost(rqb);
                cnt[cell(e, b)]--;
                const int ds = (ca1 - ca0) + (cb1 - cb0), d = kPenalty * dc + ds;
                // a tabu move is taken only if it gives a new best clash-free colouring
                if (tabu_until[(size_t)e * D + b] > it && !(clashes + dc == 0 && soft + ds < best)) continue;
                if (d < best_d) {
                    best_d = d; be = e; bc = b; ties = 1;
                } else if (d == best_d && next() % (uint64_t)(++ties) == 0) {
                    be = e; bc = b;
                }
            }
        }
        if (be < 0) break;
        const int a = col[be], u = src(be), v = tgt(be), rqa = a * nq + (u >> 3), rqb = bc * nq + (u >> 3);
        soft -= cost(rqa) + cost(rqb);
        S[u * D + a]--; R[v * D + a]--; cnt[cell(be, a)]--;
        S[u * D + bc]++; R[v * D + bc]++; cnt[cell(be, bc)]++;
        col[be] = bc;
        soft += cost(rqa) + cost(rqb);
        clashes += -((S[u * D + a] > 0) + (R[v * D + a] > 0)) + ((S[u * D + bc] > 1) + (R[v * D + bc] > 1));
        tabu_until[(size_t)be * D + a] = it + 7 + (int)(next() % 10);
        if (clashes == 0 && soft < best) {
            best = soft;
            best_col = col;
        }
    }
    col = best_col;
}

bool build_ligand(const LigandInput& in, LigandRecord& out, std::string& err) {
    const int n = in.n_atoms, nb = in.n_bonds;
    if (n < 1 || n > 64) { err = "ligand atom count must be in [1, 64]"; return false; }
    std::vector<std::vector<std::pair<int, int>>> adj(n);   // (neighbour, bond)
    for (int b = 0; b < nb; ++b) {
        const int a0 = in.bonds[2 * b], a1 = in.bonds[2 * b + 1];
        if (a0 < 0 || a1 < 0 || a0 >= n || a1 >= n || a0 == a1) { err = "bond index out of range"; return false; }
        adj[a0].push_back({a1, b});
        adj[a1].push_back({a0, b});
    }
    for (int i = 0; i < n; ++i)
        if (in.element[i] > 3) { err = "element must be 0..3 (C, N, O, S)"; return false; }
    for (int i = 0; i < 3 * n; ++i)
        if (!std::isfinite(in.xyz[i])) { err = "ligand coordinate is not finite"; return false; }
    // XS types: carbon is polar iff bonded to N or O
    out.xs.assign(n, 0);
    int type_mask = 0;
    for (int i = 0; i < n; ++i) {
        bool polar = false;
        if (in.element[i] == 0)
            for (auto& e : adj[i]) polar |= (in.element[e.first] == 1 || in.element[e.first] == 2);
        out.xs[i] = (uint8_t)xs_type(in.element[i], in.donor[i], in.acceptor[i], polar);
        type_mask |= 1 << out.xs[i];
    }
    // rigid fragments: connected components over non-rotatable bonds, numbered by lowest atom
    std::vector<int> frag(n, -1);
    int nfrag = 0;
    for (int s = 0; s < n; ++s) {
        if (frag[s] >= 0) continue;
        std::vector<int> stack{s};
        frag[s] = nfrag;
        while (!stack.empty()) {
            int a = stack.back();
            stack.pop_back();
            for (auto& e : adj[a])
                if (!in.rotatable[e.second] && frag[e.first] < 0) { frag[e.first] = nfrag; stack.push_back(e.first); }
        }
        ++nfrag;
    }
    std::vector<int> fsize(nfrag, 0);
    for (int i = 0; i < n; ++i) fsize[frag[i]]++;
    int root = 0;
    for (int f = 1; f < nfrag; ++f)
        if (fsize[f] > fsize[root]) root = f;
    int origin = -1;
    for (int i = 0; i < n && origin < 0; ++i)
        if (frag[i] == root) origin = i;
    // torsions in input order: far side = atoms cut off from the origin by the bond
    std::vector<int> rot_bonds;
    for (int b = 0; b < nb; ++b)
        if (in.rotatable[b]) rot_bonds.push_back(b);
    const int n_rot = (int)rot_bonds.size();
    if (n_rot > 26) { err = "at most 26 rotatable bonds"; return false; }
    if (nfrag > PV_MAX_FRAGS) { err = "too many rigid fragments"; return false; }
    std::vector<int> parent(nfrag, -2), ftor(nfrag, -1), anchor(nfrag, -1), near_atom(nfrag, -1);
    parent[root] = -1;
    anchor[root] = origin;
    for (int k = 0; k < n_rot; ++k) {
        const int b = rot_bonds[k];
        std::vector<char> seen(n, 0);
        std::vector<int> stack{origin};
        seen[origin] = 1;
        while (!stack.empty()) {
            int a = stack.back();
            stack.pop_back();
            for (auto& e : adj[a])
                if (e.second != b && !seen[e.first]) { seen[e.first] = 1; stack.push_back(e.first); }
        }
        const int a0 = in.bonds[2 * b], a1 = in.bonds[2 * b + 1];
        if (seen[a0] == seen[a1]) { err = "rotatable bond is not a bridge of a connected ligand"; return false; }
        const int nr = seen[a0] ? a0 : a1, fa = seen[a0] ? a1 : a0;
        const int ff = frag[fa];
        if (parent[ff] != -2) { err = "fragment reached by two rotatable bonds"; return false; }
        parent[ff] = frag[nr];
        ftor[ff] = k;
        anchor[ff] = fa;
        near_atom[ff] = nr;
    }
    for (int f = 0; f < nfrag; ++f)
        if (parent[f] == -2) { err = "ligand is not connected"; return false; }
    // depth-first preorder of fragments, children by torsion index
    std::vector<std::vector<int>> kids(nfrag);
    for (int f = 0; f < nfrag; ++f)
        if (f != root) kids[parent[f]].push_back(f);
    for (auto& k : kids) std::sort(k.begin(), k.end(), [&](int a, int b) { return ftor[a] < ftor[b]; });
    std::vector<int> order, depth(nfrag, 0);
    std::vector<int> st{root};
    while (!st.empty()) {
        int f = st.back();
        st.pop_back();
        order.push_back(f);
        for (auto it = kids[f].rbegin(); it != kids[f].rend(); ++it) {
            depth[*it] = depth[f] + 1;
            st.push_back(*it);
        }
    }
    std::vector<int> new_id(nfrag);
    for (int i = 0; i < nfrag; ++i) new_id[order[i]] = i;
    // device atom order and subtree ranges
    std::vector<int> dev_of(n), src_of;
    std::vector<int> own_start(nfrag);
    for (int fi = 0; fi < nfrag; ++fi) {
        own_start[fi] = (int)src_of.size();
        for (int i = 0; i < n; ++i)
            if (frag[i] == order[fi]) { dev_of[i] = (int)src_of.size(); src_of.push_back(i); }
    }
    auto src_of_dev = [&](int d) { return src_of[d]; };
    std::vector<int> sub_end(nfrag);
    for (int fi = nfrag - 1; fi >= 0; --fi) {
        int end = own_start[fi] + fsize[order[fi]];
        for (int c : kids[order[fi]]) end = std::max(end, sub_end[new_id[c]]);
        sub_end[fi] = end;
    }
    int max_depth = 0;
    for (int f = 0; f < nfrag; ++f) max_depth = std::max(max_depth, depth[f]);
    // intra pairs: different rigid fragments and more than three bonds apart
    std::vector<std::pair<int, int>> pairs;
    for (int i = 0; i < n; ++i) {
        std::vector<int> dist(n, -1), q{i};
        dist[i] = 0;
        for (size_t h = 0; h < q.size(); ++h)
            for (auto& e : adj[q[h]])
                if (dist[e.first] < 0) { dist[e.first] = dist[q[h]] + 1; q.push_back(e.first); }
        for (int j = i + 1; j < n; ++j)
            if (frag[i] != frag[j] && !(dist[j] >= 0 && dist[j] <= 3)) pairs.push_back({i, j});
    }
    // Schedule the pairs for the team: each pair is computed by the lane of one of its atoms (the
    // source), which keeps that atom's force in registers; the other atom's lane (the target's)
    // receives the opposite force by a shuffle from the source lane. A round gives every lane at
    // most one pair to send and one to receive, so a round needs neither atomics nor shared memory.
    // A warp schedule (32 lanes) always; a half-warp schedule (16 lanes) when the ligand fits a
    // half-warp team (at most 32 atoms, 16 fragments, 6 + n_rot <= 16 tangent coordinates).
    auto schedule = [&](int lanes, std::vector<std::vector<PvPairSlot>>& rounds) {
        std::vector<std::pair<int, int>> edges;   // (source, target), device atom indices
        for (auto& p : pairs) edges.push_back({dev_of[p.first], dev_of[p.second]});
        orient_pairs(n, edges, lanes);
        std::vector<int> colour;
        const int nr = colour_rounds(edges, colour, lanes);
        balance_banks(edges, colour, nr, lanes);
        // an empty slot sends its "pair" to the far dummy atom: beyond the cutoff, no energy, no force
        rounds.assign(nr, std::vector<PvPairSlot>(lanes, PvPairSlot{PV_DUMMY_ATOM, 0.f, 0.f, 0.f}));
        for (size_t e = 0; e < edges.size(); ++e) {
            const int src = edges[e].first, tgt = edges[e].second;
            const int ti = out.xs[src_of_dev(src)], tj = out.xs[src_of_dev(tgt)];
            const uint32_t hyd = (is_hyd(ti) && is_hyd(tj)) ? 1u : 0u;
            const uint32_t hb = ((is_don(ti) && is_acc(tj)) || (is_acc(ti) && is_don(tj))) ? 1u : 0u;
            const uint32_t half = (uint32_t)(src / lanes);
            PvPairSlot& s = rounds[colour[e]][src % lanes];
            s.meta = (int32_t)(((uint32_t)s.meta & ~127u) | (uint32_t)tgt | (half << 7) | (hyd << 16) | (hb << 17) |
                               (1u << 31));
            // the ramp w sat(c0 + c1 d): hydrophobic 1 below d = 0.5 to 0 at 1.5, H-bond 1 below
            // d = -0.7 to 0 at 0 (the two never meet in one pair)
            const float good = hyd ? kHydGood : kHBondGood, bad = hyd ? kHydBad : kHBondBad;
            s.c1 = (hyd || hb) ? -1.0f / (bad - good) : 0.0f;    // sat((bad - d) / (bad - good))
            s.c0 = (hyd || hb) ? bad / (bad - good) : 0.0f;
            s.w = hyd ? kWHydrophobic : (hb ? kWHBond : 0.0f);
            // the target's lane: which lane sends to it this round, and which of its atoms
            PvPairSlot& t = rounds[colour[e]][tgt % lanes];
            t.meta = (int32_t)((uint32_t)t.meta | ((uint32_t)(src % lanes) << 8) | (1u << 13) |
                               ((uint32_t)(tgt / lanes) << 14));
        }
        // the empty slots of a quarter-warp read the dummy atom of a residue its partners leave free
        for (auto& round : rounds)
            for (int q = 0; q < lanes; q += 8) {
                uint32_t used = 0;
                for (int l = q; l < q + 8; ++l)
                    if ((uint32_t)round[l].meta >> 31) used |= 1u << (round[l].meta & 7);
                int k = 0;
                while ((used >> k) & 1) ++k;
                for (int l = q; l < q + 8; ++l)
                    if (!((uint32_t)round[l].meta >> 31))
                        round[l].meta = (int32_t)(((uint32_t)round[l].meta & ~127u) | (uint32_t)(PV_DUMMY_ATOM + (k & 7)));
            }
        return nr;
    };
    std::vector<std::vector<PvPairSlot>> rounds, rounds16;
    const int n_rounds_sched = schedule(32, rounds);
    const bool team16 = n <= 32 && nfrag <= 16 && 6 + n_rot <= 16;
    const int n_rounds16 = team16 ? schedule(16, rounds16) : 0;
    if ((int)rounds.size() > PV_MAX_ROUNDS || n_rounds16 > 2 * PV_MAX_ROUNDS) {
        err = "intra pair schedule exceeds the round limit";
        return false;
    }
    // record
    const int n_rounds = n_rounds_sched;
    const int bytes = PV_LIG_FIXED_BYTES + (n_rounds * 32 + n_rounds16 * 16) * (int)sizeof(PvPairSlot);
    out.blob.assign((size_t)((bytes + 15) / 16) * 16, 0);
    PvLigBlob* L = reinterpret_cast<PvLigBlob*>(out.blob.data());
    L->h.n_atoms = n;
    L->h.n_rot = n_rot;
    L->h.n_frag = nfrag;
    L->h.n_pairs = (int)pairs.size();
    L->h.n_rounds = n_rounds;
    L->h.max_depth = max_depth;
    L->h.bfgs_iters = (25 + n) / 3;
    L->h.blob_bytes = (int)out.blob.size();
    L->h.origin_src = origin;
    L->h.type_mask = type_mask;
    L->h.n_rounds16 = n_rounds16;
    L->h.team16 = team16 ? 1 : 0;
    L->h.pairs16_at = n_rounds * 32;
    double g2 = 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            double d = (double)in.xyz[3 * i + k] - (double)in.xyz[3 * origin + k];
            g2 += d * d;
        }
    L->h.rgyr = (float)std::sqrt(g2 / n);
    for (int di = 0; di < n; ++di) {
        const int i = src_of[di];
        const int f = frag[i];
        const int an = anchor[f];
        int packed = new_id[f] | (out.xs[i] << 8);
        float w;
        std::memcpy(&w, &packed, 4);
        L->atom[di] = make_float4(in.xyz[3 * i] - in.xyz[3 * an], in.xyz[3 * i + 1] - in.xyz[3 * an + 1],
                                  in.xyz[3 * i + 2] - in.xyz[3 * an + 2], w);
        L->atom_src[di] = i;
    }
    for (int fi = 0; fi < nfrag; ++fi) {
        const int f = order[fi];
        const int an = anchor[f];
        int par = f == root ? 0 : new_id[parent[f]];
        float pw, dw;
        std::memcpy(&pw, &par, 4);
        int dep = depth[f];
        std::memcpy(&dw, &dep, 4);
        float ox = 0.f, oy = 0.f, oz = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
        if (f != root) {
            const int pa = anchor[parent[f]];
            ox = in.xyz[3 * an] - in.xyz[3 * pa];
            oy = in.xyz[3 * an + 1] - in.xyz[3 * pa + 1];
            oz = in.xyz[3 * an + 2] - in.xyz[3 * pa + 2];
            const int na = near_atom[f];
            double vx = (double)in.xyz[3 * an] - in.xyz[3 * na], vy = (double)in.xyz[3 * an + 1] - in.xyz[3 * na + 1],
                   vz = (double)in.xyz[3 * an + 2] - in.xyz[3 * na + 2];
            double len = std::sqrt(vx * vx + vy * vy + vz * vz);
            if (!(len > 1e-6)) { err = "rotatable bond of zero length"; return false; }
            ax = (float)(vx / len); ay = (float)(vy / len); az = (float)(vz / len);
        }
        L->frag_off[fi] = make_float4(ox, oy, oz, pw);
        L->frag_axis[fi] = make_float4(ax, ay, az, dw);
        L->frag_a0[fi] = own_start[fi];
        L->frag_a1[fi] = sub_end[fi];
        L->frag_tor[fi] = ftor[f];
        if (ftor[f] >= 0) L->tor_frag[ftor[f]] = fi;
    }
    for (int r = 0; r < n_rounds; ++r)
        for (int l = 0; l < 32; ++l) L->pairs[r * 32 + l] = rounds[r][l];
    for (int r = 0; r < n_rounds16; ++r)
        for (int l = 0; l < 16; ++l) L->pairs[n_rounds * 32 + r * 16 + l] = rounds16[r][l];
    out.n_atoms = n;
    out.n_rot = n_rot;
    out.n_pairs = (int)pairs.size();
    out.n_rounds = n_rounds;
    out.staged32 = PV_LIG_STAGED_BYTES(n_rounds, n_rounds16, 32);
    out.staged16 = PV_LIG_STAGED_BYTES(n_rounds, n_rounds16, 16);
    out.origin = origin;
    out.type_mask = type_mask;
    out.team16 = team16;
    out.subtree_atoms = 0;
    for (int fi = 1; fi < nfrag; ++fi) out.subtree_atoms += sub_end[fi] - own_start[fi];
    return true;
}

}  // namespace pv
