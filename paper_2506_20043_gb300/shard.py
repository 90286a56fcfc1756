"""Sharding of a docking job over GPUs (one process per GPU) and the host-side merge of results.

Units of the search are independent (ligand, pocket, chain), so ranks work on disjoint shards with no
data-path collective. Shards are cut by pocket first, so that each GPU builds and holds only the maps
of its own pockets, then by ligand when there are fewer pocket groups than ranks (plan_shards), or as
equal contiguous runs of the pocket-major pair list (plan_pairs: balanced to one pair, a pocket's maps
built on at most the two ranks whose runs meet inside it). Each pair keeps its random stream from the
unsplit job (its pair key), so the split does not change any chain. The only exchange
is the final one: each rank's kept poses (a few records per pair) are gathered on the host and merged
per ligand by score, ties by (pocket, chain) -- the same order the GPU merge uses within a rank.

Pocket prediction (Supplementary Algorithm 1) shards by receptor: receptors are dealt round-robin to
ranks, each rank predicts the pockets of its own receptors, and the ranked pocket lists are gathered
on one rank keyed by receptor.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

Record = Tuple[float, int, int]   # (SF, pocket id, chain)


def plan_shards(pocket_ids: Sequence[int], n_ligands: int, world: int) -> List[Tuple[List[int], List[int]]]:
    """Per rank: (pocket ids, ligand indices). Pockets are dealt round-robin to rank groups; when
    there are more ranks than pockets, the ligands of a pocket are split over the ranks sharing it."""
    if world < 1:
        raise ValueError("world must be >= 1")
    pockets = list(pocket_ids)
    if not pockets or n_ligands < 1:
        return [([], []) for _ in range(world)]
    groups = min(world, len(pockets))
    out: List[Tuple[List[int], List[int]]] = []
    for r in range(world):
        g = r % groups
        ranks_in_group = [q for q in range(world) if q % groups == g]
        k = ranks_in_group.index(r)
        my_pockets = pockets[g::groups]
        per = len(ranks_in_group)
        my_ligs = list(range(k, n_ligands, per))
        out.append((my_pockets, my_ligs))
    return out


def plan_pairs(pocket_ids: Sequence[int], n_ligands: int, world: int) -> List[List[Tuple[int, int, int]]]:
    """Per rank: its pairs as (ligand, pocket id, key), with key = ligand * len(pocket_ids) + the
    pocket's position (the pair's index, hence its random stream, in one unsplit pv_dock call). The
    job's pairs are taken pocket-major (all ligands of the first pocket, then of the next) and cut
    into `world` contiguous runs whose sizes differ by at most one, so every rank gets the same
    work to within one pair and builds the maps of only the few pockets its run touches."""
    if world < 1:
        raise ValueError("world must be >= 1")
    pockets = list(pocket_ids)
    n_p = len(pockets)
    order = [(li, pockets[k], li * n_p + k) for k in range(n_p) for li in range(max(n_ligands, 0))]
    base, extra = divmod(len(order), world)
    out, start = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append(order[start:start + size])
        start += size
    return out


def merge_records(per_rank: Sequence[Dict[int, List[Record]]]) -> Dict[int, List[Record]]:
    """Merges {ligand: [(SF, pocket, chain), ...]} from every rank into one ranking per ligand."""
    merged: Dict[int, List[Record]] = {}
    for part in per_rank:
        for lig, recs in part.items():
            merged.setdefault(lig, []).extend((float(s), int(p), int(c)) for s, p, c in recs)
    return {lig: sorted(recs) for lig, recs in merged.items()}


def records_from_result(result, ligand_ids: Sequence[int]) -> Dict[int, List[Record]]:
    """{global ligand id: records} from a DockResult of this rank (ligand_ids maps the rank's local
    ligand index to the job's ligand id). Ranks that dock their pairs with the job-wide pair keys
    (pv_dock_params.pair_keys) and the same search team width reproduce, after merge_records, the
    ranking of one unsplit dock bit for bit."""
    poses = result.poses.reshape(-1)
    out: Dict[int, List[Record]] = {}
    for local, lig in enumerate(ligand_ids):
        out[int(lig)] = [(float(poses[i]["score"]), int(poses[i]["pocket"]), int(poses[i]["chain"]))
                         for i in result.ranking(local)]
    return out


def gather_merge(local: Dict[int, List[Record]], group=None, dst: int = 0):
    """Gathers every rank's records on rank `dst` (torch.distributed, any backend) and merges them
    there; other ranks get None."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    bucket = [None] * world if rank == dst else None
    dist.gather_object(local, bucket, dst=dst, group=group)
    return merge_records(bucket) if rank == dst else None


Pocket = Tuple[float, float, float, float, int]   # (Eq. 2 score, centre x, y, z, points)


def plan_receptors(n_receptors: int, world: int) -> List[List[int]]:
    """Per rank: the receptor indices it predicts pockets for (round-robin)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    return [list(range(r, max(n_receptors, 0), world)) for r in range(world)]


def pockets_from_clusters(clusters) -> List[Pocket]:
    """The ranked pockets of one receptor from its Clusters (best first)."""
    c = clusters.read()
    return [(float(s), float(x[0]), float(x[1]), float(x[2]), int(n))
            for s, x, n in zip(c["score"], c["center"], c["size"])]


def gather_pockets(local: Dict[int, List[Pocket]], group=None, dst: int = 0):
    """Gathers every rank's {receptor: ranked pockets} on rank `dst` (torch.distributed, any
    backend); other ranks get None. Receptors are disjoint across ranks, so this is a union."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    bucket = [None] * world if rank == dst else None
    dist.gather_object(local, bucket, dst=dst, group=group)
    if rank != dst:
        return None
    out: Dict[int, List[Pocket]] = {}
    for part in bucket:
        for rec, pockets in part.items():
            if int(rec) in out:
                raise ValueError(f"receptor {rec} predicted on two ranks")
            out[int(rec)] = [tuple(p) for p in pockets]
    return dict(sorted(out.items()))
