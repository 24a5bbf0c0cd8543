"""Target-row partition of a suspension across ranks (host logic).

The matvec shards by target rows: each rank owns a contiguous run of whole
bodies (so the body-block preconditioner stays rank-local), receives every
source position and force (one all-gather per matvec) and computes its own rows
with no reduction.  On a one-GPU-per-box deployment the bench runs replicas;
this module is the partition a multi-GPU run would use.
"""


def body_ranges(nb: int, world: int):
    """Split bodies 0..nb-1 into `world` contiguous ranges whose sizes differ by
    at most one body (equal rows, hence equal pair work per rank)."""
    if nb < 0 or world < 1:
        raise ValueError("nb >= 0 and world >= 1 required")
    base, extra = divmod(nb, world)
    out, b0 = [], 0
    for rank in range(world):
        b1 = b0 + base + (1 if rank < extra else 0)
        out.append((b0, b1))
        b0 = b1
    return out


def blob_ranges(nb: int, nper: int, world: int):
    """The blob (row) ranges of body_ranges."""
    return [(b0 * nper, b1 * nper) for b0, b1 in body_ranges(nb, world)]
