"""Several GPUs on one MLMC estimate: a sample-range dispenser.

Samples are independent (Sec. 2.2, Remark 3.3), so ranks share the work of
every sampling phase. Each level's missing samples are dispensed as
contiguous index ranges sized by the batch rule of Eq. (batch)
(``mlmc_batch_size``), levels finest first (the priority of Algorithm 1):
an idle rank claims the next range with one atomic add on a shared
key-value store, so no rank waits for a coordinator. A rank solves its
ranges on its own GPU. At the end of the phase the per-sample values
(Q_l, Q_{l-1}) are all-gathered (16 bytes per sample) and every rank folds
all of them, level by level in index order, into its plan's level states:
each rank then holds the state a single GPU would have built, bit for bit,
computes the same allocation (Eq. (mlmc_num_samples)) and the same
estimate, whatever the number of ranks or the order in which ranges were
claimed.

``run_rounds`` is the same exchange with one graph-captured round per rank
and phase (shares fixed by Eq. (batch) with every rank claiming once), so
the latency-bound coarse levels of a rank's share overlap its fine ones as
in the single-GPU run; ``tensor_gather`` moves the values as one float64
all-gather (NCCL between GPUs).

The data path has one exchange per phase (the all-gather); everything
else is local. ``run_sharded`` is transport-agnostic: the store, the
all-gather and the per-rank sampler/fold/allocation callables are passed
in, so the same code runs over NCCL/gloo process groups on GPUs and over
gloo on CPUs in tests.
"""
from . import mlmc as _m

PHI_INV = 0.6180339887498949


class RangeDispenser:
    """Claims contiguous ranges of one phase's missing samples from a store.

    ``store`` needs ``add(key, amount) -> new value`` (atomic), as
    ``torch.distributed.TCPStore`` provides."""

    def __init__(self, store, parts, prefix="mlmc", min_frac=0.01, max_frac=PHI_INV):
        self.store, self.parts, self.prefix = store, parts, prefix
        self.min_frac, self.max_frac = min_frac, max_frac

    def claim(self, phase, level, first, count):
        """Next range (start, size) of [first, first + count) for this rank, or None."""
        key = "%s/%d/%d" % (self.prefix, phase, level)
        while True:
            n = int(self.store.add(key, 0))
            if n >= count:
                return None
            b = _m.batch_size(count, n, self.parts, self.min_frac, self.max_frac)
            end = int(self.store.add(key, b))
            start = end - b
            if start >= count:
                return None
            return first + start, min(b, count - start)


def run_sharded(n_levels, sample, fold, reset, allocate, all_gather, dispenser, eps=None,
                pilot=0, N_fixed=None, max_phases=64):
    """Adaptive MLMC (Sec. 2.3, L fixed) over several ranks.

    sample(level, first, count) -> (qf, qc) sequences for those samples;
    reset() clears the local level states; fold(level, qf, qc) folds values
    in the order given; allocate(eps) -> N_l per level from the local states;
    all_gather(obj) -> list of every rank's obj. Returns (N per level, the
    ranges this rank solved as (phase, level, first, count))."""
    have = [0] * n_levels
    target = list(N_fixed) if N_fixed is not None else [pilot] * n_levels
    history = [dict() for _ in range(n_levels)]   # first index -> (qf, qc)
    claimed = []
    for phase in range(max_phases):
        mine = []
        for l in range(n_levels - 1, -1, -1):
            count = target[l] - have[l]
            while count > 0:
                got = dispenser.claim(phase, l, have[l], count)
                if got is None:
                    break
                first, size = got
                qf, qc = sample(l, first, size)
                mine.append((l, first, [float(x) for x in qf], [float(x) for x in qc]))
                claimed.append((phase, l, first, size))
        for part in all_gather(mine):
            for l, first, qf, qc in part:
                history[l][first] = (qf, qc)
        reset()
        for l in range(n_levels):
            qf_all, qc_all, nxt = [], [], 0
            for first in sorted(history[l]):
                if first != nxt:
                    raise RuntimeError("level %d: samples %d..%d missing after the gather"
                                       % (l, nxt, first - 1))
                qf, qc = history[l][first]
                qf_all += qf
                qc_all += qc
                nxt = first + len(qf)
            if nxt != target[l]:
                raise RuntimeError("level %d: %d samples gathered, %d expected" % (l, nxt, target[l]))
            if qf_all:
                fold(l, qf_all, qc_all)
        have = list(target)
        if N_fixed is not None or phase == max_phases - 1:
            break
        need = allocate(eps)
        more = False
        for l in range(n_levels):
            if need[l] > target[l]:
                target[l] = int(need[l])
                more = True
        if not more:
            break
    return have, claimed


def plan_callables(plan):
    """sample / fold / reset / allocate for run_sharded on one GPU plan."""
    import numpy as np

    def sample(level, first, count):
        qf, qc, _ = plan.sample_level(level, first, count)
        return qf, (qc if level > 0 else np.zeros_like(qf))

    def fold(level, qf, qc):
        plan.level_fold(level, qf, qc if level > 0 else None)

    return sample, fold, plan.reset_stats, plan.allocation


def shares(missing, world):
    """Contiguous shares of one level's missing samples, one per rank: the
    batch of Eq. (batch) with every rank claiming once, b = ceil(missing /
    world); rank r takes [r b, min((r + 1) b, missing)). Returns (start, size)
    relative to the first missing sample, for every rank."""
    b = -(-missing // world) if missing > 0 else 0
    out = []
    for r in range(world):
        lo = min(r * b, missing)
        out.append((lo, min(lo + b, missing) - lo))
    return out


def run_rounds(plan, rank, world, gather, eps=None, pilot=0, N_fixed=None, max_phases=64):
    """Adaptive MLMC (Sec. 2.3, L fixed) over `world` ranks, one round per rank
    per sampling phase.

    In every phase each level's missing samples are split into contiguous
    shares (``shares``); a rank runs its share of every level as one
    graph-captured round (``plan.round``: a branch per level), reads the
    round's per-sample values back (16 bytes per sample) and ``gather``s
    them; every rank then folds all values of every level in index order
    into its plan's level states (``plan.reset_stats``, ``plan.level_fold``),
    so each rank holds the level states a single GPU builds for the same
    samples, bit for bit, and computes the same allocation. ``gather(counts,
    values)`` receives this rank's values (one float64 array per level: its
    Q_l then its Q_{l-1}) and the counts of every rank and level
    (counts[r][l]), and returns the arrays of every rank in rank order.

    Returns (N per level, estimate, sum_l V_l / N_l) from the plan."""
    import numpy as np
    L1 = plan.cfg.n_levels
    have = [0] * L1
    target = [int(x) for x in N_fixed] if N_fixed is not None else [int(pilot)] * L1
    hist_f = [np.zeros(0) for _ in range(L1)]
    hist_c = [np.zeros(0) for _ in range(L1)]
    for phase in range(max_phases):
        part = [shares(target[l] - have[l], world) for l in range(L1)]
        counts = [[part[l][r][1] for l in range(L1)] for r in range(world)]
        first = [have[l] + part[l][rank][0] for l in range(L1)]
        mine = counts[rank]
        vals = [np.zeros(0) for _ in range(L1)]
        in_round = False
        if sum(mine):
            try:
                plan.round(first, mine)
                in_round = True
            except _m.MLMCError as e:
                # the round does not fit the workspace together: level by level
                if e.status != _m.MLMC_ERR_UNIMPLEMENTED:
                    raise
        for l in range(L1):
            if not mine[l]:
                continue
            if in_round:
                qf, qc = plan.round_values(l, mine[l])
            else:
                qf, qc, _ = plan.sample_level(l, first[l], mine[l])
                qc = qc if l > 0 else np.zeros_like(qf)
            vals[l] = np.concatenate([qf, qc])
        every = gather(counts, vals)
        for l in range(L1):
            fs, cs = [hist_f[l]], [hist_c[l]]
            for r in range(world):
                c = counts[r][l]
                fs.append(every[r][l][:c])
                cs.append(every[r][l][c:2 * c])
            hist_f[l] = np.concatenate(fs)
            hist_c[l] = np.concatenate(cs)
        plan.reset_stats()
        for l in range(L1):
            if hist_f[l].size:
                plan.level_fold(l, hist_f[l], hist_c[l] if l > 0 else None)
        have = list(target)
        if N_fixed is not None:
            break
        need = plan.allocation(eps)
        more = False
        for l in range(L1):
            if need[l] > target[l]:
                target[l] = int(need[l])
                more = True
        if not more:
            break
    q, v = plan.estimate()
    return have, q, v


def tensor_gather(dist, device):
    """``gather`` for run_rounds over a torch.distributed process group: the
    values of every rank travel in one all_gather_into_tensor of float64 (NCCL
    on GPUs, gloo on CPUs); the receiving side splits them by the counts every
    rank already knows."""
    import numpy as np
    import torch

    def gather(counts, vals):
        world = len(counts)
        sizes = [2 * sum(c) for c in counts]
        width = max(1, max(sizes))
        mine = np.concatenate(vals) if vals else np.zeros(0)
        buf = torch.zeros(width, dtype=torch.float64, device=device)
        if mine.size:
            buf[:mine.size] = torch.from_numpy(mine).to(device)
        out = torch.empty(world * width, dtype=torch.float64, device=device)
        dist.all_gather_into_tensor(out, buf)
        host = out.cpu().numpy().reshape(world, width)
        every = []
        for r in range(world):
            arrs, o = [], 0
            for c in counts[r]:
                arrs.append(host[r, o:o + 2 * c].copy())
                o += 2 * c
            every.append(arrs)
        return every

    return gather
