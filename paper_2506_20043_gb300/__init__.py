"""GB300-native docking hot path of PocketVina (arxiv 2506.20043).

Per-pocket receptor grid maps, Vina-style pose scoring with its adjoint gradient, and batched
Monte-Carlo + RILC-BFGS search over every ligand x pocket pair, in hand-written sm_103a CUDA
behind the C ABI of include/pocketvina.h. ``build()`` compiles the library in-tree; the API
(``Context``, ``DockParams``, ``PVScore``, ``PVScoreXYZ``) lives in ``api``.
"""
from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Context", "DockParams", "PVScore", "PVScoreXYZ", "PVError", "GridSet", "Ligand", "DockResult"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
