"""GB300-native node2vec second-order random walks (GRAPE, arXiv 2110.06196).

The compute path is libgrape_walk (CUDA, sm_103a) behind the C ABI declared in
include/grape_walk.h; ``walk`` is its Python face (argument marshalling over
ctypes), and ``elias_fano`` that of the Elias-Fano graph store.  ``synth``
builds seeded synthetic inputs.
"""
from .walk import (BatchPlan, Graph, Server, autotune_batched, contexts, contexts_from_rows,
                   philox4x32_10, sector_probe, walks, walks_approx, walks_batched, walks_cumsum,
                   walks_host)
from .elias_fano import EFGraph, ef_walks
from ._lib import GrapeError

__all__ = ["Graph", "walks", "walks_cumsum", "walks_approx", "walks_host", "walks_batched", "BatchPlan", "autotune_batched",
           "Server", "contexts", "contexts_from_rows", "philox4x32_10", "sector_probe",
           "EFGraph", "ef_walks", "GrapeError"]
