"""Host-side plan of one trajectory split over several GPUs by orbitals (columns of U).

The paper runs each trajectory on one device (App. A); a lattice whose U and propagator
exceed one GPU's memory would need the orbitals spread over R ranks.  Rank r holds the
columns [lo_r, hi_r) of U (L x N_r).  One step then needs these exchanges and no others:

  propagation   U_r <- P U_r                         local (P replicated, or its stencil)
  occupations   n_i = sum_r sum_{k in r} |U_ik|^2    all-reduce of an L-vector (sum)
  QSD weight    U_r <- diag(w(n, xi)) U_r             local (same Philox draws on every rank)
  Gram          G[:, r] = U^dag U_r                  all-gather of the column blocks of U, then
                                                     an all-reduce of N x N (each rank adds its
                                                     block column into zeros)
  factor        R, T = R^-1 of G                     replicated on every rank (same G, same result)
  product       U_r <- U T[:, r]                     local, on the gathered U
  projective    p_j = sum_r |U_{j, r}|^2             all-reduce of a scalar per event,
  event         v = sum_r U_r conj(x_r)^T            and of an L-vector
  entropy       C_A = sum_r U_{A, r} U_{A, r}^dag    all-reduce of |A| x |A|

This module holds only that plan: the shard ranges and the collectives (torch.distributed,
any backend).  The arithmetic between them is the single-GPU library's kernels applied to a
column block; the multi-GPU path is not built for GPUs (each box here has one) and its
communication is unmeasured on hardware.  Its exchanges are checked with gloo ranks on the
CPU (tests/test_split_plan.py), where the test supplies the local arithmetic.
"""


def column_shards(N, world, align=128):
    """Balanced [lo, hi) column ranges of N orbitals over `world` ranks, boundaries on
    multiples of `align` where N allows (the tensor-core tiles are 128 wide)."""
    if world < 1 or N < world:
        raise ValueError("need 1 <= world <= N")
    unit = align if N % align == 0 and N // align >= world else 1
    blocks = N // unit
    out, lo = [], 0
    for r in range(world):
        nb = blocks // world + (1 if r < blocks % world else 0)
        hi = lo + nb * unit
        out.append((lo, hi))
        lo = hi
    return out


class SplitPlan:
    """The exchanges of one split trajectory for this rank (torch.distributed initialised)."""

    def __init__(self, L, N, world=None, rank=None, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group) if world is None else world
        self.rank = dist.get_rank(group) if rank is None else rank
        self.L, self.N = L, N
        self.shards = column_shards(N, self.world)
        self.lo, self.hi = self.shards[self.rank]

    @property
    def ncols(self):
        return self.hi - self.lo

    def bytes_per_step(self, elem=8, events=0, ee_sites=0):
        """Bytes each rank sends per step (ring collectives: 2 (R-1)/R of an all-reduce's
        buffer, (R-1)/R of an all-gather's), for complex elements of `elem` bytes."""
        R = self.world
        f = (R - 1) / R
        b = 2 * f * 8 * self.L                          # occupations (float64)
        b += f * elem * self.L * self.N                 # gather of U
        b += 2 * f * elem * self.N * self.N             # Gram
        b += events * 2 * f * (8 + elem * self.L)       # projective events
        b += 2 * f * elem * ee_sites * ee_sites         # entropy
        return b

    def allreduce_occupations(self, partial):
        """partial: this rank's sum_{k in r} |U_ik|^2 (tensor of L); returns n_i in place."""
        self.dist.all_reduce(partial, op=self.dist.ReduceOp.SUM, group=self.group)
        return partial

    def gather_columns(self, U_local):
        """The full U (L x N, columns in rank order) from every rank's block (L x N_r)."""
        import torch
        parts = [torch.empty((self.L, hi - lo), dtype=U_local.dtype, device=U_local.device)
                 for (lo, hi) in self.shards]
        self.dist.all_gather(parts, U_local.contiguous(), group=self.group)
        return torch.cat(parts, dim=1)

    def allreduce_gram(self, G_cols):
        """G_cols: this rank's block column U^dag U_r (N x N_r); returns the full N x N G."""
        import torch
        G = torch.zeros((self.N, self.N), dtype=G_cols.dtype, device=G_cols.device)
        G[:, self.lo:self.hi] = G_cols
        self.dist.all_reduce(G, op=self.dist.ReduceOp.SUM, group=self.group)
        return G

    def allreduce_sum(self, x):
        """Sum over ranks in place (the Born weight, v = U x^dag, C_A)."""
        self.dist.all_reduce(x, op=self.dist.ReduceOp.SUM, group=self.group)
        return x
