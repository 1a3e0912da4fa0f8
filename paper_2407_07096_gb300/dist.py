"""Multi-GPU exact KDE (one process per GPU, torch.distributed).

The sum over points shards naturally (Sec. 3: K(q) = sum_i k(||q - x_i||) over the
whole point set):
  * by data: rank r holds the contiguous block ``shard_range(n, r, world)`` of X and
    computes the partial sums of every query on its GPU; one FP64 all-reduce (SUM) of
    the m partials gives K on every rank. The normalised density divides by the global n.
  * by query (replicas): every rank holds all of X and evaluates its own slice of the
    query rows; no exchange is needed unless the caller wants the full vector
    (``gather_rows``).
All arithmetic stays in the library's kernels; this module only moves FP64 vectors.
"""
from __future__ import annotations


def shard_range(count: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block [lo, hi) of ``count`` items owned by ``rank`` of ``world``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    lo = count * rank // world
    hi = count * (rank + 1) // world
    return lo, hi


def allreduce_partials(partials, group=None):
    """Sums per-shard FP64 partial densities across ranks (in place) and returns them."""
    import torch
    import torch.distributed as dist
    if partials.dtype != torch.float64:
        raise ValueError("partials must be float64")
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(partials, op=dist.ReduceOp.SUM, group=group)
    return partials


def gather_rows(local, m_total, group=None):
    """Concatenates every rank's contiguous slice of a length-``m_total`` FP64 vector."""
    import torch
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return local
    world = dist.get_world_size(group)
    sizes = [shard_range(m_total, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    buf = torch.zeros(width, dtype=local.dtype, device=local.device)
    buf[: local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[: hi - lo] for p, (lo, hi) in zip(parts, sizes)])


def _backend(group):
    import torch.distributed as dist
    if not (dist.is_initialized() and dist.get_world_size(group) > 1):
        return None
    return str(dist.get_backend(group)).lower()


class ShardedExactKDE:
    """Data-sharded exact KDE: this rank's GPU holds only its block of X.

    ``query`` / ``query_dev`` evaluate every query against the local block (the library's
    kernels) and sum the per-rank FP64 partials with one all-reduce. Under NCCL the
    partials stay on the device and the all-reduce runs on the device tensor; under gloo
    (host collectives) they are moved to host memory for the exchange and back.
    ``local_factory(X_block, a, **kw)`` builds the per-rank evaluator (default: the
    library's ExactGaussianKDE); it must offer ``query(Q) -> float64 array`` and, for
    ``query_dev``, ``query_dev(Q, out)``.
    """

    def __init__(self, X, a: float, rank: int, world: int, normalise: bool = False, local_factory=None, **kw):
        self.n_total = int(X.shape[0])
        lo, hi = shard_range(self.n_total, rank, world)
        if hi <= lo:
            raise ValueError("every rank needs at least one point")
        if local_factory is None:
            from .kde import ExactGaussianKDE as local_factory
        self.local = local_factory(X[lo:hi], a, **kw)
        self.block = (lo, hi)
        self.normalise = normalise

    def _scaled(self, tot):
        return tot / self.n_total if self.normalise else tot

    def query_dev(self, Q, out=None, group=None, stream=None):
        """Densities of the rows of the CUDA tensor Q as a CUDA float64 tensor (every rank
        receives all m values). Synchronises ``stream`` before the exchange."""
        import torch
        part = self.local.query_dev(Q, out, stream) if stream is not None else self.local.query_dev(Q, out)
        backend = _backend(group)
        if backend is None:
            return self._scaled(part)
        (stream or torch.cuda.current_stream(part.device)).synchronize()
        if backend == "nccl":
            allreduce_partials(part, group)
            return self._scaled(part)
        host = allreduce_partials(part.cpu(), group)
        part.copy_(host)
        return self._scaled(part)

    def query(self, Q, group=None):
        """Densities of the rows of the host array Q (float64 numpy array on every rank)."""
        import numpy as np
        import torch
        backend = _backend(group)
        if backend == "nccl":
            dev = torch.device("cuda", torch.cuda.current_device())
            dt = getattr(self.local, "_np_dtype", np.float32)
            Qd = torch.from_numpy(np.ascontiguousarray(Q, dtype=dt)).to(dev)
            return self.query_dev(Qd, group=group).cpu().numpy()
        part = torch.from_numpy(np.asarray(self.local.query(Q), dtype=np.float64).copy())
        tot = allreduce_partials(part, group)
        return self._scaled(tot).numpy()

    def close(self):
        self.local.close()
