// pv_ligand.h -- host-side ligand record construction (torsion tree, pairs, schedule).
#pragma once
#include <stdint.h>
#include <string>
#include <vector>

#include "pv_layout.h"

namespace pv {

struct LigandInput {
    int n_atoms;
    const float* xyz;
    const uint8_t* element;
    const uint8_t* donor;
    const uint8_t* acceptor;
    int n_bonds;
    const int32_t* bonds;
    const uint8_t* rotatable;
};

struct LigandRecord {
    std::vector<uint8_t> blob;   // PvLigBlob followed by the pair rounds, 16-byte padded
    std::vector<uint8_t> xs;     // XS type per input atom
    int n_atoms = 0, n_rot = 0, n_pairs = 0, n_rounds = 0, origin = 0, type_mask = 0;
    int staged32 = 0, staged16 = 0;   // bytes of the record staged for a warp / half-warp team
    int subtree_atoms = 0;       // sum over torsions of the atoms each one moves
    bool team16 = false;         // fits a half-warp team
};

bool build_ligand(const LigandInput& in, LigandRecord& out, std::string& err);

}  // namespace pv
