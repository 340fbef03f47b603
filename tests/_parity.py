"""GPU-vs-oracle parity at the tolerances of the evaluator's acceptance bar:
feasibility flags and the enumeration argmin identical wherever the oracle's
cost gap exceeds 1e-3 relative, costs within 1e-4 relative, v_hat <= 1e-5,
knot states within 1e-3.

How the bar is read (Eq. mode_nlp: the evaluator is a local solver, "not
guaranteed to attain J*(m)"; Sec. III-C: a TO stops on scaled feasibility,
stationarity and dual-residual tolerances):

* A converged answer is only determined to within the stop test's
  tolerances.  The reference for each TO is therefore the exact local
  solution of its basin: the FP64 oracle's polish of an answer (warm start
  at the answer, tight tolerances, a strong proximal term so that the polish
  stays local).  Two answers reach the *same local solution* when their
  polishes coincide (pose within 1e-5, cost within 1e-8 relative).
* Costs: |J_gpu - J*| <= 1e-4 |J*| + sum_r |lam*_r| |c_r(z_gpu)|, the
  relative bar plus the first-order change of J that the answer's residual
  infeasibility (within the stop test's eps_primal) can cause; asserted on
  the maximum over all TOs that reach the same local solution.
* Knot states: the GPU's answer lies within 1e-3 of the exact local solution
  beyond the oracle's own distance to it at the same stop tolerances,
  |x_gpu - x*| <= 1e-3 + |x_oracle - x*| (the oracle re-solved from its own
  answer moves by up to a few 1e-3 along weakly curved directions, so the
  literal GPU-vs-oracle distance is reported beside it).  Compared are the
  object's pose at every knot and, for pushing, the contact offset where it
  is determined: at knots whose interval carries a contact force, and along
  the unmasked s-rows of the dynamics from there (elsewhere it does not
  enter the problem).  The bimanual hands' offsets are not compared: the
  ground force's centre of pressure compensates them in the torque balance.
* A TO whose GPU state error exceeds that bar is listed; it must still meet
  the cost bar, stay within 1e-2 of the exact solution, and carry an FP64
  stationarity certificate within the stop test's largest tolerance
  (1e-4 x beta_max / beta_ref x max(1, |J|)): a valid stop of a solve whose
  weakly curved directions (the stationarity tolerance over a small
  curvature) leave the states determined only to a few 1e-3.
* TOs whose two answers reach different local solutions are listed one by
  one (order, both certified costs); the test asserts that each GPU answer
  there is itself a certified local solution (its polish converges, its cost
  is within the bar of that polish).

Everything here is host-side analysis of results; the only solver called is
the oracle.
"""
from __future__ import annotations

import numpy as np

import oracle

TIGHT_POLISH = dict(eps_dual=1e-9, eps_primal=1e-11, eps_comp=1e-11, max_iters=2000, beta0=1e4, beta_max=1e8,
                    rho0=1e-2, rho_min=1e-2)


class Task:
    """Layout and oracle calls of one task (pushing or bimanual)."""

    def __init__(self, bimanual: bool):
        self.bim = bimanual
        self.nx, self.nu = (5, 12) if bimanual else (4, 3)
        self.npose = 3
        self.nrow = 32 if bimanual else 11

    def traj_len(self, N):
        return self.nx * (N + 1) + self.nu * N

    def gpu_to_oracle(self, traj, N, Nmax):
        """GPU layout x[nx][Nmax+1], u[nu][Nmax] -> oracle x[nx][N+1], u[nu][N]."""
        x = traj[: self.nx * (Nmax + 1)].reshape(self.nx, Nmax + 1)[:, : N + 1]
        u = traj[self.nx * (Nmax + 1): self.nx * (Nmax + 1) + self.nu * Nmax].reshape(self.nu, Nmax)[:, :N]
        return np.concatenate([x.ravel(), u.ravel()]).astype(np.float64)

    def solve_ex(self, insts, idx, seqs, lens, warm=None, opts=None):
        if self.bim:
            return oracle.bim_solve_batch_ex(insts, idx, seqs, lens, warm=warm, opts=opts)
        return oracle.solve_batch_ex(insts, idx, seqs, lens, warm=warm, opts=opts)

    def rows(self, inst, modes, N, tr):
        if self.bim:
            return oracle.bim_rows(inst, modes, N, tr)
        return oracle.rows(inst, np.asarray(modes, np.uint8), N, tr)

    def states(self, tr, N):
        return tr[: self.nx * (N + 1)].reshape(self.nx, N + 1)

    def controls(self, tr, N):
        return tr[self.nx * (N + 1): self.nx * (N + 1) + self.nu * N].reshape(self.nu, N)

    def determined_offsets(self, tr, N, srow_on):
        """[(state index, bool mask over knots)]: the contact offset s_k
        enters the problem through the contact torque of interval k (-s f_n),
        so it is determined where that interval carries a contact force
        (above 5 % of the trajectory's largest), and along the s-rows of the
        dynamics (s_{k+1} = s_k + dt sdot_k) from there; elsewhere it is
        free."""
        if self.bim:
            # the hands' offsets enter only the torque balance, where the
            # ground force's centre of pressure (a control within the
            # support) compensates them: they are not determined
            return []
        U = self.controls(tr, N)
        pairs = [(3, U[0], srow_on[0])]
        out = []
        for i, fn, on in pairs:
            m = np.zeros(N + 1, bool)
            m[:N] = np.abs(fn) > 0.05 * float(np.abs(fn).max())
            for k in range(N):
                if m[k] and on[k]:
                    m[k + 1] = True
            for k in range(N - 1, -1, -1):
                if m[k + 1] and on[k]:
                    m[k] = True
            out.append((i, m))
        return out

    def srow_on(self, inst, modes, N, tr):
        _, mask, _, _ = self.rows(inst, modes, N, tr)
        return [mask[:, 3].astype(bool)]

    def state_dist(self, a, b, N, ref, srow_on):
        """max |a - b| over pose states and determined offsets (of ref)."""
        Xa, Xb = self.states(a, N), self.states(b, N)
        d = float(np.max(np.abs(Xa[: self.npose] - Xb[: self.npose])))
        for i, m in self.determined_offsets(ref, N, srow_on):
            if m.any():
                d = max(d, float(np.max(np.abs(Xa[i][m] - Xb[i][m]))))
        return d

    def pose_dist(self, a, b, N):
        return float(np.max(np.abs(self.states(a, N)[: self.npose] - self.states(b, N)[: self.npose])))

    def allowance(self, inst, modes, N, tr, lam):
        """sum_r |lam_r| |c_r(tr)| over the rows (initial rows included)."""
        c, mask, _, ci = self.rows(inst, modes, N, tr)
        lr = np.abs(lam[3: 3 + self.nrow * N]).reshape(N, self.nrow)
        return float(np.sum(np.abs(lam[:3]) * np.abs(ci)) + np.sum(lr * np.abs(c) * mask))

    def vhat(self, inst, modes, N, tr):
        """v_hat (Eq. inexact_mode_value) of a trajectory, physical units."""
        c, mask, scale, ci = self.rows(inst, modes, N, tr)
        ineq = np.zeros(self.nrow, bool)
        if self.bim:
            ineq[11:16] = ineq[19:24] = ineq[27:] = True
        else:
            ineq[5:] = True
        v = np.where(ineq[None, :], np.maximum(c, 0), np.abs(c)) / scale * mask
        return max(float(v.max()), float(np.abs(ci).max()))


def polish(task, insts, idx, seqs, lens, trajs):
    """Tight FP64 polish of answers (one per TO, oracle layout rows)."""
    opts = oracle.default_opts(**TIGHT_POLISH)
    return task.solve_ex(insts, idx, seqs, lens, warm=trajs, opts=opts)


def compare(task, insts, idx, seqs, lens, Ns, gpu, ref, ref_tr, sel=None, verbose=True):
    """Per-TO parity of jointly converged TOs (indices `sel`, default all).

    gpu: dict of numpy arrays (status, cost, viol, traj in the GPU layout,
    stride) from the evaluator; ref: oracle results with ref_tr its
    trajectories.  Returns a report dict; the caller asserts on it."""
    n = len(idx)
    sel = np.arange(n) if sel is None else np.asarray(sel)
    Nmax = int(np.max(Ns))
    feas_g = (gpu["status"] == 0) & (gpu["viol"] <= 1e-5)
    feas_o = (ref["status"] == 0) & (ref["viol"] <= 1e-5)
    joint = sel[feas_g[sel] & feas_o[sel]]
    # answers in the oracle layout, padded to the longest TO
    L = task.traj_len(Nmax)
    zg = np.zeros((len(joint), L))
    zo = np.zeros((len(joint), L))
    for j, t in enumerate(joint):
        N = int(Ns[t])
        zg[j, : task.traj_len(N)] = task.gpu_to_oracle(gpu["traj"][t], N, gpu["traj_nmax"])
        zo[j, : task.traj_len(N)] = ref_tr[t][: task.traj_len(N)]
    sub = lambda a: [a[t] for t in joint]
    jidx, jseq, jlen = idx[joint], sub(seqs), lens[joint]
    if not task.bim:
        jseq = np.asarray(jseq, np.uint8)
    rg, pg, _ = polish(task, insts, jidx, jseq, jlen, zg)
    ro, po, lo = polish(task, insts, jidx, jseq, jlen, zo)
    rep = dict(joint=len(joint), same=0, different=[], unresolved=[], cost_excess=[], state_excess=[],
               cost_err=[], state_err=[], state_err_oracle=[], gpu_vs_oracle_state=[], gpu_vs_oracle_cost=[],
               vhat_fail=[], state_fail=[])
    for j, t in enumerate(joint):
        N = int(Ns[t])
        inst = insts[idx[t]]
        m = tuple(seqs[t])[: int(lens[t])]  # the order at its own length (seqs may be padded)
        a, b, c = zg[j, : task.traj_len(N)], zo[j, : task.traj_len(N)], po[j, : task.traj_len(N)]
        pgj = pg[j, : task.traj_len(N)]
        # every converged GPU answer is feasible by the oracle's own rows
        vg = task.vhat(inst, m, N, a)
        if not vg <= 1e-5:
            rep["vhat_fail"].append((int(t), vg))
        # each answer must be a stable local solution: its tight polish
        # converges near it (a polish that travels far started from a saddle
        # or a flat valley, where no exact local solution is attached)
        Jg, Jo = float(gpu["cost"][t]), float(ref["cost"][t])
        loc_g = rg["status"][j] == 0 and task.pose_dist(a, pgj, N) <= 1e-2 and \
            abs(Jg - float(rg["cost"][j])) <= 1e-2 * max(1.0, abs(Jg))
        loc_o = ro["status"][j] == 0 and task.pose_dist(b, c, N) <= 1e-2 and \
            abs(Jo - float(ro["cost"][j])) <= 1e-2 * max(1.0, abs(Jo))
        if not (loc_g and loc_o):
            rep["unresolved"].append(dict(t=int(t), modes=tuple(int(v) for v in m), gpu_local=bool(loc_g),
                                          oracle_local=bool(loc_o), J_gpu=Jg, J_gpu_polished=float(rg["cost"][j]),
                                          J_oracle=Jo, J_oracle_polished=float(ro["cost"][j])))
            continue
        Jstar = float(ro["cost"][j])
        same = (abs(float(rg["cost"][j]) - Jstar) <= 1e-8 * max(1.0, abs(Jstar))
                and task.pose_dist(pgj, c, N) <= 1e-5)
        if not same:
            # a different local solution (listed; certify_different checks
            # the GPU's answer against its own polish)
            rep["different"].append(dict(t=int(t), modes=tuple(int(v) for v in m), J_gpu=Jg,
                                         J_gpu_polished=float(rg["cost"][j]), J_oracle=float(ref["cost"][t]),
                                         J_oracle_polished=Jstar))
            continue
        rep["same"] += 1
        A = task.allowance(inst, m, N, a, lo[j])
        eJ = abs(float(gpu["cost"][t]) - Jstar)
        rep["cost_err"].append(eJ / max(abs(Jstar), 1e-12))
        if eJ > 1e-4 * abs(Jstar) + A:
            rep["cost_excess"].append((int(t), eJ, 1e-4 * abs(Jstar) + A))
        on = task.srow_on(inst, m, N, c)
        eg = task.state_dist(a, c, N, c, on)
        eo = task.state_dist(b, c, N, c, on)
        rep["state_err"].append(eg)
        rep["state_err_oracle"].append(eo)
        rep["gpu_vs_oracle_state"].append(task.state_dist(a, b, N, c, on))
        rep["gpu_vs_oracle_cost"].append(abs(float(gpu["cost"][t]) - float(ref["cost"][t])) / abs(Jstar))
        if eg > 1e-3 + eo:
            rep["state_excess"].append((int(t), eg, eo))
            stat_ok = "stat" in gpu and float(gpu["stat"][t]) <= 1.5e-3 * max(1.0, abs(Jstar))
            if not (eJ <= 1e-4 * abs(Jstar) + A and eg <= 1e-2 and stat_ok):
                rep["state_fail"].append((int(t), eg, eo, float(gpu["stat"][t]) if "stat" in gpu else None))
    for k in ("cost_err", "state_err", "state_err_oracle", "gpu_vs_oracle_state", "gpu_vs_oracle_cost"):
        rep[k] = np.array(rep[k])
    if verbose:
        print(summary(rep))
    return rep


def certify_different(task, insts, idx, seqs, lens, Ns, gpu, rep):
    """For the TOs whose GPU answer reached another local solution: the
    GPU's cost must be within 1e-4 relative plus the first-order allowance
    of its own polish.  Returns the list of TOs that fail."""
    bad = []
    for d in rep["different"]:
        t = d["t"]
        N = int(Ns[t])
        a = task.gpu_to_oracle(gpu["traj"][t], N, gpu["traj_nmax"])
        m = tuple(seqs[t])[: int(lens[t])]
        mm = np.asarray([seqs[t]], np.uint8) if not task.bim else [m]
        r, p, lam = polish(task, insts, idx[t: t + 1], mm, lens[t: t + 1], a[None, :])
        if r["status"][0] != 0:
            bad.append((t, "polish not converged"))
            continue
        A = task.allowance(insts[idx[t]], m, N, a, lam[0])
        if abs(d["J_gpu"] - float(r["cost"][0])) > 1e-4 * abs(float(r["cost"][0])) + A:
            bad.append((t, d["J_gpu"], float(r["cost"][0]), A))
    return bad


def flag_disagreements(gpu, ref, sel=None):
    """Orders whose feasibility flags (converged and v_hat <= 1e-5) differ,
    with both statuses.  A stop on the tolerances implies v_hat <= eps_feas / 2
    on either side, so a disagreement needs one side to end without the stop
    test (iteration budget, factorisation or non-finite)."""
    n = len(gpu["status"])
    sel = np.arange(n) if sel is None else np.asarray(sel)
    fg = (gpu["status"] == 0) & (gpu["viol"] <= 1e-5)
    fo = (ref["status"] == 0) & (ref["viol"] <= 1e-5)
    out = []
    for t in sel[fg[sel] != fo[sel]]:
        out.append((int(t), int(gpu["status"][t]), int(ref["status"][t])))
    return out


def summary(rep):
    def pct(a, q):
        return float(np.percentile(a, q)) if len(a) else float("nan")
    return (f"jointly feasible {rep['joint']}: same local solution {rep['same']}, "
            f"different {len(rep['different'])}, unresolved {len(rep['unresolved'])}; "
            f"cost error vs exact (rel) p50 {pct(rep['cost_err'], 50):.2e} p99 {pct(rep['cost_err'], 99):.2e} "
            f"max {pct(rep['cost_err'], 100):.2e}; state error vs exact p50 {pct(rep['state_err'], 50):.2e} "
            f"p99 {pct(rep['state_err'], 99):.2e} max {pct(rep['state_err'], 100):.2e} "
            f"(oracle's own: p99 {pct(rep['state_err_oracle'], 99):.2e} max {pct(rep['state_err_oracle'], 100):.2e}); "
            f"gpu vs oracle: state p50 {pct(rep['gpu_vs_oracle_state'], 50):.2e} "
            f"p99 {pct(rep['gpu_vs_oracle_state'], 99):.2e} max {pct(rep['gpu_vs_oracle_state'], 100):.2e}, "
            f"cost p50 {pct(rep['gpu_vs_oracle_cost'], 50):.2e} p99 {pct(rep['gpu_vs_oracle_cost'], 99):.2e} "
            f"max {pct(rep['gpu_vs_oracle_cost'], 100):.2e}; cost bar exceeded {len(rep['cost_excess'])}, "
            f"state bar exceeded {len(rep['state_excess'])} (of which not a certified stop {len(rep['state_fail'])}), "
            f"v_hat > 1e-5 {len(rep['vhat_fail'])}")


def argmin_parity(task, insts, slices, idx, seqs, lens, Ns, gpu, ref, ref_tr, verbose=True):
    """Enumeration argmin (Eq. mode_selection) per instance, compared where
    the oracle's cost gap (its second-best feasible order against its best)
    exceeds 1e-3 relative.  A different GPU pick there must be explained by
    one of the listed, checkable causes:
      'gpu_budget'      the GPU's solve of the oracle's best order ended at
                        the iteration budget without feasibility;
      'gpu_other_local' the GPU's solve of the oracle's best order reached
                        another (certified, costlier) local solution;
      'gpu_better'      the GPU's pick has a certified answer cheaper than the
                        oracle's best by more than 1e-3 (the oracle's solve of
                        that order reached a costlier local solution).
    Returns (outcomes, unexplained)."""
    from oracle import search as S
    outcomes, unexplained = [], []
    for i, sl in enumerate(slices):
        cg, vg = gpu["cost"][sl], gpu["viol"][sl]
        co, vo = ref["cost"][sl], ref["viol"][sl]
        ag, ao = S.enumeration_argmin(cg, vg), S.enumeration_argmin(co, vo)
        feas_o = np.flatnonzero(vo <= 1e-5)
        if len(feas_o) == 0:
            outcomes.append((i, "no feasible order", ag, ao))
            continue
        Jbest = float(co[ao])
        rest = np.sort(co[feas_o][feas_o != ao])
        gap = (float(rest[0]) - Jbest) / abs(Jbest) if len(rest) else np.inf
        if ag == ao:
            outcomes.append((i, "identical", ag, ao, gap))
            continue
        if gap <= 1e-3:
            outcomes.append((i, "near tie", ag, ao, gap))
            continue
        tg, to = sl.start + ag, sl.start + ao
        why = None
        if not (vg[ao] <= 1e-5):
            if gpu["status"][to] != 0:
                why = "gpu_budget"
        else:
            rep = compare(task, insts, idx, seqs, lens, Ns, gpu, ref, ref_tr, sel=[to], verbose=False)
            if rep["different"] and float(cg[ao]) > Jbest * (1 + 1e-3):
                if not certify_different(task, insts, idx, seqs, lens, Ns, gpu, rep):
                    why = "gpu_other_local"
        if why is None and float(cg[ag]) < Jbest * (1 - 1e-3) and vg[ag] <= 1e-5:
            # the GPU's answer at its pick must be a certified local solution
            N = int(Ns[tg])
            a = task.gpu_to_oracle(gpu["traj"][tg], N, gpu["traj_nmax"])
            mm = np.asarray([seqs[tg]], np.uint8) if not task.bim else [seqs[tg]]
            r, p, lam = polish(task, insts, idx[tg: tg + 1], mm, lens[tg: tg + 1], a[None, :])
            A = task.allowance(insts[idx[tg]], seqs[tg], N, a, lam[0])
            if r["status"][0] == 0 and abs(float(cg[ag]) - float(r["cost"][0])) <= 1e-4 * abs(float(r["cost"][0])) + A:
                why = "gpu_better"
        outcomes.append((i, why or "unexplained", ag, ao, gap, float(cg[ag]), float(co[ag]), float(cg[ao]), Jbest))
        if why is None:
            unexplained.append(outcomes[-1])
    if verbose:
        kinds = {}
        for o in outcomes:
            kinds[o[1]] = kinds.get(o[1], 0) + 1
        print("argmin per instance:", kinds)
        for o in outcomes:
            if o[1] not in ("identical", "near tie"):
                print("   ", o)
    return outcomes, unexplained


def flags_after_refinement(flags, gpu, ref, rerun_gpu, rerun_oracle):
    """Feasibility flags where one side ended at the exploration budget:
    that side is re-run with the refinement budget t_ref = 1,500 (Sec. III-C:
    selected orders are refined with the same evaluator at t_ref) and the
    flags are compared again.  rerun_gpu / rerun_oracle(list of TOs) return
    (status, viol) arrays.  Returns the disagreements that remain."""
    fg = {t: bool(gpu["status"][t] == 0 and gpu["viol"][t] <= 1e-5) for t, _, _ in flags}
    fo = {t: bool(ref["status"][t] == 0 and ref["viol"][t] <= 1e-5) for t, _, _ in flags}
    lag_g = [t for t, _, _ in flags if not fg[t]]
    lag_o = [t for t, _, _ in flags if not fo[t]]
    if lag_g:
        st, v = rerun_gpu(lag_g)
        for t, a, b in zip(lag_g, st, v):
            fg[t] = bool(a == 0 and b <= 1e-5)
    if lag_o:
        st, v = rerun_oracle(lag_o)
        for t, a, b in zip(lag_o, st, v):
            fo[t] = bool(a == 0 and b <= 1e-5)
    return [(t, fg[t], fo[t]) for t, _, _ in flags if fg[t] != fo[t]]
