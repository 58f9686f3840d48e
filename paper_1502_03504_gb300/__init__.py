"""GB300-native library for the hot path of locally-oriented programming (LOPe).

A local function writes one array element and reads a fixed-width halo around
it (Rasmussen et al., arXiv:1502.03504, Sec. 2); the library applies it at
every point of a 2D/3D structured grid for many time steps.  All computation
runs in the CUDA kernels of ``liblope.so`` (sm_103a) behind a C ABI
(``include/lope.h``); this package only marshals arguments.  PyTorch supplies
device memory and streams.

The ``lope_*`` functions mirror the C ABI one to one; ``Grid``, ``Stencil``
and the helpers below wrap them for torch tensors.
"""
from ._lib import (  # noqa: F401
    BC_DIRICHLET,
    BC_PERIODIC,
    DTYPES,
    LopeError,
    SCHEMES,
    Grid,
    Launch,
    Stencil,
    apply,
    apply_batch,
    apply_host,
    plan,
    adjoint,
    autotune,
    autotune_batch,
    batch_workspace_size,
    forward_ckpt,
    launch_count,
    library_path,
    load,
    reduce_sum,
    reduce_sqdiff,
    sync_status,
    version,
    vjp,
    workspace_size,
)
from ._lib import (  # noqa: F401  (C ABI names)
    lope_adjoint,
    lope_apply,
    lope_apply_host,
    lope_apply_batch,
    lope_apply_with,
    lope_autotune,
    lope_autotune_batch,
    lope_batch_workspace_size,
    lope_forward_ckpt,
    lope_grid_create,
    lope_grid_destroy,
    lope_last_error,
    lope_launch_count,
    lope_reduce,
    lope_reduce_noalloc,
    lope_reduce_scratch_bytes,
    lope_set_option,
    lope_set_boundary,
    lope_stencil_create_builtin,
    lope_stencil_compile,
    lope_stencil_create_linear,
    lope_stencil_create_source,
    lope_stencil_destroy,
    lope_stencil_set_scheme,
    lope_plan,
    lope_sync_status,
    lope_tune_cache_load,
    lope_tune_cache_save,
    lope_version,
    lope_vjp,
    lope_work_states,
    lope_workspace_size,
)
