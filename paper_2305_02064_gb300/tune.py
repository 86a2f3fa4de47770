"""Autotuner of the gridding form and launch shape.

Every setting of ``mmsar_tiles`` computes the same image (the FP32 shapes
bit for bit, the grouped and the tensor-core forms to FP32 rounding); which
is fastest depends on the scan (the tensor-core form wherever the tiles hold
enough samples; among the FP32 forms a small scan fills the GPU better with
CTAs over 32 frequencies or 8 x 8-cell tiles, a large one prefers 64 or 128
frequencies; arrays whose pairs share x offsets gain from the grouped form).  ``autotune`` images the caller's own data with each shape on
the caller's stream, timed with CUDA events, and leaves the plan set to the
fastest; the result is kept on the plan, so plans shared by scans of one
shape are tuned once.  Only the plan's launch shape changes: the kernels
and the images are the library's.
"""
from __future__ import annotations

# (frequencies per lane, warps per CTA, grouped, tensor cores): the
# tensor-core form, then the FP32 forms (four frequencies per lane: 4 x 2-cell
# warp blocks, per-sample form only)
TENSOR_CORES = tuple((2, 4, 0, v) for v in (5, 2, 1, 3, 4))   # the pipeline variants
SHAPES = (TENSOR_CORES + tuple((nf, wp, gr, 0) for gr in (1, 0) for nf, wp in ((2, 8), (1, 8), (2, 4), (1, 4)))
          + ((4, 8, 0, 0), (4, 4, 0, 0)))


def autotune(plan, ws, echo, pos, tx, rx, vol, echo_scale=None, stream=None, reps: int = 3,
             shapes=SHAPES) -> dict:
    """Time ``reps`` images per launch shape (after one untimed image) and set
    the fastest on ``plan``.  Returns {"tiles": (nf, warps, grouped, tc), "ms": {shape: ms}}.
    Grouped shapes are skipped when the plan rejects them (too many Tx/Rx pairs)."""
    import torch
    st = stream or torch.cuda.current_stream(vol.device)
    from ._lib import MmsarError
    times = {}
    for shp in shapes:
        try:
            plan.set_tiles(*shp)
        except MmsarError:
            continue
        plan.image(ws, echo, pos, tx, rx, vol, echo_scale=echo_scale, stream=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            plan.image(ws, echo, pos, tx, rx, vol, echo_scale=echo_scale, stream=st)
        e1.record(st)
        e1.synchronize()
        times[shp] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    plan.set_tiles(*best)
    plan.tuned = {"tiles": best, "ms": times}
    return plan.tuned
