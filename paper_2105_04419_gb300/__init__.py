"""GB300-native exact truncated Euclidean distance transform over a sparse brick grid.

Python binding of ``libvdbedt.so`` (C ABI in ``include/vdbedt.h``).  Argument marshalling only:
every step of the transform runs in the library's CUDA kernels.  PyTorch provides device memory
and streams.  The library must be built (``paper_2105_04419_gb300.build.build()``); without it,
importing :mod:`paper_2105_04419_gb300.lib` raises.

Entry points mirror the C names: :class:`Map` wraps a handle (create, set_occupancy,
set_occupancy_counted, set_occupancy_dense, reset, global_, update, query, export_dense, clearance_forward /
clearance_backward, set_tuning, synchronize, info); :class:`UpdateGraph` captures one
incremental update into a CUDA graph and replays it per frame (:class:`GlobalGraph` the same for
the global transform from fresh records); :class:`Batch` holds grids
of uneven size whose transform steps run once for all of them; :func:`global_batched` runs
several maps in one call; :func:`clearance_cost` is the differentiable clearance cost (torch.autograd.Function
over the library's forward and backward kernels).
"""
from .lib import (  # noqa: F401
    Batch,
    BatchUpdateGraph,
    D_NONE,
    GlobalGraph,
    VDBEDT_DMAX_LIMIT,
    Map,
    UpdateGraph,
    VdbedtError,
    brick_masks,
    clearance_cost,
    edt_dense_noalloc,
    global_batched,
    kernel_launches,
    pack_records,
    UNBOUNDED_MAX,
    UNBOUNDED_MIN,
    UNBOUNDED_OFFSET,
    library_path,
    load,
)
