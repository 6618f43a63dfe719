"""List-mode MLEM of one job over several ranks (one GPU per rank).

Event sharding (sharded_mlem):

Each rank keeps its shard of the events resident in its own context, with the
same grid and the same sensitivity image.  An iteration is one event pass per
rank (recon_event_pass), one sum of the C images over the ranks (an all-reduce,
the only exchange of the iteration) and the same update on every rank
(recon_update), so every rank holds the same image after every iteration.  The
backprojection C_j = sum_i a_ij w_i / p_i is a sum over events, so the sum of the
ranks' C is the C of the whole list and the iteration is MLEM over all events
(Sec. 2.4); only the order of the FP32 sums differs.  The first pass starts
from the image 1 on {s_j > 0}: MLEM's first update from any uniform image is the
same, so the ranks need not agree on a start value.

Region sharding (region_block, regions_mlem_sharded): the body regions of the
TOF-assisted division (Sec. 2.5) are reconstructed independently, so each rank
takes a consecutive block of them, reconstructs its slabs, and the whole-body
image is the sum of the ranks' stitched images (each holds only its own slabs):
one sum at the end, no exchange between iterations.
"""


def sharded_mlem(ctx, n_iter, c_buf, allreduce_sum, image_out=None):
    """n_iter MLEM iterations of this rank's context in step with the other ranks.

    ctx: a binding.Context with this rank's events resident and the sensitivity
    set.  c_buf: nx*ny*nz float32 buffer (host or device, wherever allreduce_sum
    works).  allreduce_sum(c_buf, n_eff) sums c_buf over the ranks in place and
    returns the summed n_eff.  Returns [(N_eff, sum_j s_j lambda_j)] per iteration
    (both over all ranks' events)."""
    history = []
    for k in range(n_iter):
        n_eff = ctx.event_pass(None, None, 1 if k == 0 else 0, c_buf)
        n_eff = allreduce_sum(c_buf, n_eff)
        ssum = ctx.update(c_buf, image_out if k == n_iter - 1 else None)
        history.append((n_eff, ssum))
    return history


def torch_allreduce_sum(group=None):
    """allreduce_sum over a torch.distributed process group (NCCL with device
    buffers, gloo with host buffers)."""
    import torch
    import torch.distributed as dist

    def fn(c_buf, n_eff):
        dist.all_reduce(c_buf, group=group)
        t = torch.tensor([float(n_eff)], dtype=torch.float64, device=c_buf.device)
        dist.all_reduce(t, group=group)
        return float(t.item())

    return fn


def region_block(n_regions, rank, world):
    """The consecutive regions [lo, hi) of rank `rank` (blocks as equal as the
    count allows; a rank may get none when there are more ranks than regions)."""
    lo = rank * n_regions // world
    hi = (rank + 1) * n_regions // world
    return lo, hi


def regions_mlem_sharded(ctx, regions, margin_mm, shell_mm, n_iter, image, rank, world, allreduce_image):
    """This rank's block of the regions, reconstructed and stitched into `image`
    (nx*ny*nz float32, zero outside its slabs), then summed over the ranks by
    allreduce_image(image).  The division passed to the library is the whole one,
    so events shared with a region of another rank keep their weight 1/2.
    Returns the block (lo, hi)."""
    lo, hi = region_block(len(regions), rank, world)
    if hi > lo:
        ctx.set_region_block(lo, hi - lo)
        try:
            ctx.mlem_regions(None, regions, margin_mm, shell_mm, n_iter, image)
        finally:
            ctx.set_region_block(0, 0)
    else:
        image.zero_() if hasattr(image, "zero_") else image.fill(0)
    allreduce_image(image)
    return lo, hi
