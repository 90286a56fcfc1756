// Test harness (host only): builds a ligand record with the library's host-side builder and
// decodes its intra-pair schedules, so the CPU tests can check them against the oracle's pair
// list without a GPU.
#include <string>

#include "pv_ligand.h"

extern "C" int lig_schedule(int n_atoms, const float* xyz, const uint8_t* el, const uint8_t* don,
                            const uint8_t* acc, int n_bonds, const int32_t* bonds, const uint8_t* rot,
                            int lanes, int32_t* out, int max_out, int32_t* info) {
    pv::LigandInput in{n_atoms, xyz, el, don, acc, n_bonds, bonds, rot};
    pv::LigandRecord rec;
    std::string err;
    if (!pv::build_ligand(in, rec, err)) return -1;
    const PvLigBlob* L = reinterpret_cast<const PvLigBlob*>(rec.blob.data());
    info[0] = L->h.n_rounds;
    info[1] = L->h.n_rounds16;
    info[2] = L->h.team16;
    info[3] = L->h.n_pairs;
    if (lanes != 32 && lanes != 16) return -2;
    const int rounds = lanes == 32 ? L->h.n_rounds : L->h.n_rounds16;
    const uint32_t* w0 = L->pairs + (lanes == 32 ? 0 : L->h.n_rounds * 32);
    int k = 0;
    for (int r = 0; r < rounds; ++r)
        for (int l = 0; l < lanes; ++l) {
            const uint32_t w = w0[r * lanes + l];
            if (!(w >> 31)) continue;
            if (k >= max_out) return -3;
            const int src = l + lanes * (int)((w >> 6) & 1u), tgt = (int)(w & 63u);
            out[6 * k + 0] = r;
            out[6 * k + 1] = l;
            out[6 * k + 2] = src < L->h.n_atoms ? L->atom_src[src] : -1;
            out[6 * k + 3] = tgt < L->h.n_atoms ? L->atom_src[tgt] : -1;
            out[6 * k + 4] = (int)((w >> 16) & 1u);
            out[6 * k + 5] = (int)((w >> 17) & 1u);
            ++k;
        }
    return k;
}
