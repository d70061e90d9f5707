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
