"""Oracle: the scheduling pieces of the paper, in plain Python.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Eq. (batch) (Sec. 4): the next batch of a level is a contiguous range of
  sample indices. The printed formula is garbled (as printed it is always 1);
  the text says the batch follows the unassigned share (N - n) / N, bounded
  by fractions (1% and 1/phi) of the per-partition share ceil(N / parts).
  Reading: b = ceil((N - n) / parts) clamped to
  [max(1, ceil(0.01 s)), max(1, floor(s / phi))], s = ceil(N / parts), and
  at most N - n.
* Algorithm 1 (Sec. 3): tasks needing q_l processors, q_0 | q_1 | ... | q_L
  | p, scheduled finest level first, each task to the group of q_l
  processors with the least workload (the group that becomes free first;
  ties: lowest group index). Tasks may be dispensed in batches by a serial
  coordinator that spends a fixed time per dispatch (Sec. 4 and the "Pause"
  model of Sec. 5.1).
* Theorem 3.1: under the divisibility hypothesis no processor idles before
  the last task starts, so the makespan is below W_LB + max task <= 2 W_LB.
"""
import math

PHI_INV = 2.0 / (1.0 + math.sqrt(5.0))


def batch_size(N, n, parts, min_frac=0.01, max_frac=PHI_INV):
    """Eq. (batch) as read above (0 when the level is exhausted)."""
    if n >= N:
        return 0
    share = -(-N // parts)
    b = -(-(N - n) // parts)
    lo = max(1, math.ceil(min_frac * share))
    hi = max(1, math.floor(max_frac * share))
    return min(max(b, lo), hi, N - n)


def batches(N, parts, min_frac=0.01, max_frac=PHI_INV):
    """The contiguous ranges (first, count) that Eq. (batch) cuts [0, N) into."""
    out, n = [], 0
    while n < N:
        b = batch_size(N, n, parts, min_frac, max_frac)
        out.append((n, b))
        n += b
    return out


def greedy(q, n_tasks, w, p, batch=False, min_frac=0.01, max_frac=PHI_INV, dispatch_cost=0.0):
    """Simulate Algorithm 1. w: per level, a list of task times.

    Returns dict(makespan, work_total, work_lb, last_start, idle_before_last,
    batches) and the start time of every task (levels in index order)."""
    L = len(q)
    work_total = 0.0
    for l in range(L):
        s = 0.0
        for x in w[l]:
            s += x
        work_total += q[l] * s
    fin = [0.0] * p
    starts = [[0.0] * n_tasks[l] for l in range(L)]
    idle = coord = big = last = 0.0
    count = 0
    for l in range(L - 1, -1, -1):
        G = p // q[l]
        assigned = 0
        while assigned < n_tasks[l]:
            best, ready_best = 0, None
            for g in range(G):
                ready = max(fin[g * q[l]:(g + 1) * q[l]])
                if ready_best is None or ready < ready_best:
                    best, ready_best = g, ready
            b = batch_size(n_tasks[l], assigned, G, min_frac, max_frac) if batch else 1
            coord = max(coord, ready_best) + dispatch_cost
            s = coord
            t = s
            for j in range(assigned, assigned + b):
                starts[l][j] = t
                t += w[l][j]
            big = max(big, t - s)
            last = max(last, s)
            for k in range(best * q[l], (best + 1) * q[l]):
                idle += s - fin[k]
                fin[k] = t
            assigned += b
            count += 1
    makespan = max(fin)
    for k in range(p):
        if fin[k] < last:
            idle += last - fin[k]
    return dict(makespan=makespan, work_total=work_total,
                work_lb=max(work_total / p, big), last_start=last,
                idle_before_last=idle, batches=count), starts


def optimal_makespan(w, p):
    """Brute-force optimum for single-processor tasks (tiny instances)."""
    best = math.inf
    n = len(w)

    def rec(i, loads):
        nonlocal best
        if max(loads) >= best:
            return
        if i == n:
            best = max(loads)
            return
        seen = set()
        for k in range(p):
            if loads[k] in seen:
                continue
            seen.add(loads[k])
            loads[k] += w[i]
            rec(i + 1, loads)
            loads[k] -= w[i]

    rec(0, [0.0] * p)
    return best


def pause_times(rng, mu, var, n):
    """Sec. 5.1 "Pause" model: n task times uniform on mu -/+ sqrt(3 var)."""
    a = math.sqrt(3.0 * var)
    return [rng.uniform(mu - a, mu + a) for _ in range(n)]
