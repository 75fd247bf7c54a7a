"""GB300-native EIC single-source shortest paths (arXiv 2506.19349).

The compute path is libeic (CUDA, sm_103a) behind the C ABI in include/eic.h;
``binding`` is a thin ctypes layer over it and ``graphgen`` produces seeded
synthetic inputs.
"""
from .binding import (EIC_INF, FLAG_NO_FUSE, FLAG_NO_PULL, STEP_PULL, STEP_SWEPT, Batch, EicError, Graph, Params, Server,
                      default_params, load_library, new_dist, sssp, sssp_batch, sssp_noalloc, strerror, to_host_u32)

__all__ = ["EIC_INF", "FLAG_NO_FUSE", "FLAG_NO_PULL", "STEP_PULL", "STEP_SWEPT", "Batch", "EicError", "Graph", "Params", "Server", "default_params",
           "load_library", "new_dist", "sssp", "sssp_batch", "sssp_noalloc", "strerror", "to_host_u32"]
