// Test harness (host only): builds a ligand record with the library's host-side builder and
// returns its intra-pair schedule words, so the CPU tests can check them against the oracle's pair
// list without a GPU.
#include <string>

#include "pv_ligand.h"

// Copies the schedule of the given team width (32 or 16 lanes): the meta word of each slot,
// words[r * lanes + l], and the input
// index of every device atom. info = n_rounds, n_rounds16, team16, n_pairs, n_atoms. Returns the
// number of rounds copied, or a negative code.
extern "C" int lig_schedule(int n_atoms, const float* xyz, const uint8_t* el, const uint8_t* don,
                            const uint8_t* acc, int n_bonds, const int32_t* bonds, const uint8_t* rot,
                            int lanes, uint32_t* words, int max_words, int32_t* atom_src, int32_t* info) {
    pv::LigandInput in{n_atoms, xyz, el, don, acc, n_bonds, bonds, rot};
    pv::LigandRecord rec;
    std::string err;
    if (!pv::build_ligand(in, rec, err)) return -1;
    const PvLigBlob* L = reinterpret_cast<const PvLigBlob*>(rec.blob.data());
    info[0] = L->h.n_rounds;
    info[1] = L->h.n_rounds16;
    info[2] = L->h.team16;
    info[3] = L->h.n_pairs;
    info[4] = L->h.n_atoms;
    if (lanes != 32 && lanes != 16) return -2;
    const int rounds = lanes == 32 ? L->h.n_rounds : L->h.n_rounds16;
    if (rounds * lanes > max_words) return -3;
    const PvPairSlot* w0 = L->pairs + (lanes == 32 ? 0 : L->h.n_rounds * 32);
    for (int i = 0; i < rounds * lanes; ++i) words[i] = (uint32_t)w0[i].meta;
    for (int a = 0; a < L->h.n_atoms; ++a) atom_src[a] = L->atom_src[a];
    return rounds;
}
