"""Fused Harris pattern pipeline for one B300 GPU (sm_103a).

The data-parallel computation a RISE/Shine-style compiler produces from map, zip, reduce,
slide2D and pad patterns -- gray -> 3x3 Sobel -> gradient products -> 3x3 box sum ->
det - kappa * trace^2 -- as hand-written CUDA kernels behind the C ABI of include/shine.h
(libshine.so), with a torch.autograd.Function over the hand-written adjoint kernel and a
persistent, graph-capturable batched path.

Every call fails loudly (ImportError) when libshine.so is missing: there is no CPU or library
fallback. Build it with ``python -m paper_2201_03611_b300.build``.
"""
from ._lib import LIB_PATH, ShineError, lib  # noqa: F401
from .batched import BatchedPlan  # noqa: F401
from .ops import (HarrisFn, bwd_workspace_bytes, corners, harris, harris_window, iterate_stencil,  # noqa: F401
                  iterate_sum, mv, output_shape, pipeline_bwd, pipeline_fwd, pipeline_fwd_bwd, stencil2d)
