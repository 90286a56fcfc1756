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
    // schedule into rounds: each round holds <= 32 pairs and no atom twice (first fit)
    std::vector<std::vector<uint32_t>> rounds;
    std::vector<std::vector<char>> used;
    for (auto& p : pairs) {
        const int i = dev_of[p.first], j = dev_of[p.second];
        const int ti = out.xs[p.first], tj = out.xs[p.second];
        const uint32_t hyd = (is_hyd(ti) && is_hyd(tj)) ? 1u : 0u;
        const uint32_t hb = ((is_don(ti) && is_acc(tj)) || (is_acc(ti) && is_don(tj))) ? 1u : 0u;
        const uint32_t w = (uint32_t)i | ((uint32_t)j << 8) | (hyd << 16) | (hb << 17) | (1u << 31);
        size_t r = 0;
        while (r < rounds.size() && (rounds[r].size() >= 32 || used[r][i] || used[r][j])) ++r;
        if (r == rounds.size()) { rounds.emplace_back(); used.emplace_back(64, 0); }
        rounds[r].push_back(w);
        used[r][i] = used[r][j] = 1;
    }
    if ((int)rounds.size() > PV_MAX_ROUNDS) { err = "intra pair schedule exceeds the round limit"; return false; }
    // record
    const int n_rounds = (int)rounds.size();
    const int bytes = PV_LIG_FIXED_BYTES + n_rounds * 32 * 4;
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
        for (size_t l = 0; l < rounds[r].size(); ++l) L->pairs[r * 32 + l] = rounds[r][l];
    out.n_atoms = n;
    out.n_rot = n_rot;
    out.n_pairs = (int)pairs.size();
    out.n_rounds = n_rounds;
    out.origin = origin;
    out.type_mask = type_mask;
    out.subtree_atoms = 0;
    for (int fi = 1; fi < nfrag; ++fi) out.subtree_atoms += sub_end[fi] - own_start[fi];
    return true;
}

}  // namespace pv
