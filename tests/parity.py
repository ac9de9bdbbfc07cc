"""Parity checks of GPU eigenpairs against the oracle (reading of the
tolerances: residual, eigenvalue and per-cluster subspace angle)."""
import numpy as np

from oracle.laplacian import Laplacian


def all_pairs(g):
    """Every eigenpair of L on the complement of e by the dense definition
    (graphs small enough for a dense eigensolve): no cluster can run past
    the end of this list."""
    from oracle import dense
    return dense.smallest_eigpairs(g, g.n - 1)


def clusters(ev: np.ndarray, gap: float):
    """Group consecutive sorted eigenvalues whose spacing is below `gap`."""
    groups, cur = [], [0]
    for i in range(1, ev.size):
        if ev[i] - ev[i - 1] < gap:
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups


def check_eigpairs(g, ev, V, ev_ref, V_ref, tol=1e-8, ev_rtol=1e-7, angle=1e-6, k=None):
    """ev, V: k GPU pairs; ev_ref, V_ref: at least k oracle pairs.  A cluster
    that holds one of the first k pairs must end before the oracle's list
    does (a spacing above the threshold), unless the list is the whole
    spectrum on the complement of e; otherwise the check fails and asks for
    more oracle pairs.

    * explicit FP64 residual ||L v - ev v|| <= tol ||L||_1 (recomputed here)
    * V orthonormal and orthogonal to e
    * |ev - ev_ref| <= ev_rtol |ev_ref| (absolute ev_rtol ||L||_1 near zero)
    * per cluster (Davis-Kahan: spacing below max||r|| / angle), the largest
      principal angle between the GPU vectors of the cluster and the oracle's
      cluster span is below `angle`
    """
    lap = Laplacian(g)
    k = k or ev.size
    ev, V = np.asarray(ev)[:k], np.asarray(V)[:, :k]
    R = lap.matvec(V) - V * ev[None, :]
    rn = np.linalg.norm(R, axis=0)
    assert rn.max() <= tol * lap.norm1, f"residual {rn.max() / lap.norm1:.3e} > {tol}"
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-8, "not orthonormal"
    assert np.abs(V.sum(axis=0)).max() <= 1e-8 * np.sqrt(g.n), "not orthogonal to e"
    err = np.abs(ev - ev_ref[:k])
    ref = np.abs(ev_ref[:k])
    bound = np.where(ref > 1e-9 * lap.norm1, ev_rtol * ref, ev_rtol * 1e-3 * lap.norm1)
    assert np.all(err <= bound), f"eigenvalue error {err.max():.3e} (rel {np.max(err / np.maximum(np.abs(ev_ref[:k]), 1e-300)):.3e})"
    gap = max(rn.max(), 1e-300) / angle
    worst = 0.0
    for cl in clusters(np.asarray(ev_ref), gap):
        idx = [i for i in cl if i < k]
        if not idx:
            continue
        if cl[-1] >= ev_ref.size - 1 and ev_ref.size < g.n - 1:
            # the cluster runs to the end of the oracle's list, which is not
            # the whole spectrum on the complement of e: eigenvalues beyond
            # the list may belong to it, so its span is unknown
            raise AssertionError(
                f"cluster {cl[0]}..{cl[-1]} reaches the end of the {ev_ref.size} oracle pairs "
                f"(spacing threshold {gap:.3e}): compute more oracle pairs")
        U = V_ref[:, cl]
        Vc = V[:, idx]
        s = np.linalg.norm(Vc - U @ (U.T @ Vc), ord=2)
        worst = max(worst, s)
    assert worst <= angle, f"cluster subspace angle {worst:.3e} > {angle}"
    return dict(max_rel_residual=rn.max() / lap.norm1, max_ev_rel_err=float(np.max(err / np.maximum(np.abs(ev_ref[:k]), 1e-300))),
                max_angle=worst)


def check_against_values(g, ev, V, ev_ref, tol=1e-8, ev_rtol=1e-7, angle=1e-6):
    """Parity at sizes where the oracle's vectors are not kept: ev_ref holds
    the m smallest eigenvalues on the complement of e (m > k, ascending, from
    the oracle), V the k GPU vectors.

    * explicit FP64 residual ||L v - ev v|| <= tol ||L||_1, V orthonormal, V
      orthogonal to e;
    * completeness and values: the k GPU values are the k smallest of ev_ref
      within ev_rtol (nothing below them was missed, by the oracle's order);
    * subspace angle per cluster without vectors (Davis-Kahan sin-theta): the
      GPU vectors of a cluster of eigenvalues (spacing below max||r|| / angle)
      are within ||R_c||_F / gap of the true eigenspace, gap = the distance
      from the GPU values to the nearest eigenvalue outside the cluster; the
      bound must be below `angle`.  When a cluster runs past the end of the
      stored list the residual cannot separate it from eigenvalues beyond the
      list and no per-cluster angle is certified (angle_bound None; on
      power-law graphs, whose ||L||_1 is a thousand times their smallest
      eigenvalues, this is the rule at 1e-8 ||L||_1);
    * the whole k-dimensional subspace: if the largest GPU value lies below
      the (k+1)-th stored eigenvalue, span(V) is within ||R||_F / gap of the
      span of the k smallest eigenvectors (subspace_bound)."""
    lap = Laplacian(g)
    k = ev.size
    R = lap.matvec(V) - V * ev[None, :]
    rn = np.linalg.norm(R, axis=0)
    assert rn.max() <= tol * lap.norm1, f"residual {rn.max() / lap.norm1:.3e} > {tol}"
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-8, "not orthonormal"
    assert np.abs(V.sum(axis=0)).max() <= 1e-8 * np.sqrt(g.n), "not orthogonal to e"
    assert ev_ref.size > k, "need more stored values than pairs"
    err = np.abs(ev - ev_ref[:k])
    rel = err / np.abs(ev_ref[:k])
    assert np.all(rel <= ev_rtol), f"eigenvalue error {rel.max():.3e}"
    gapc = max(rn.max(), 1e-300) / angle
    worst = 0.0
    for cl in clusters(ev_ref, gapc):
        idx = [i for i in cl if i < k]
        if not idx:
            continue
        if cl[-1] >= ev_ref.size - 1:
            worst = None
            break
        lo = ev_ref[cl[0] - 1] if cl[0] > 0 else -np.inf
        hi = ev_ref[cl[-1] + 1]
        th = ev[idx]
        gap = min(th.min() - lo, hi - th.max())  # the GPU values to the spectrum outside the cluster
        worst = max(worst, np.linalg.norm(R[:, idx]) / gap)
    if worst is not None:
        assert worst <= angle, f"certified cluster angle {worst:.3e} > {angle}"
    sub = np.linalg.norm(R) / (ev_ref[k] - ev.max()) if ev.max() < ev_ref[k] else None
    return dict(max_rel_residual=rn.max() / lap.norm1, max_ev_rel_err=float(rel.max()), angle_bound=worst,
                subspace_bound=sub, residual_fro=float(np.linalg.norm(R)))


def subspace_sin(U, W):
    """Largest principal-angle sine between span(U) and span(W) (orthonormal
    columns, same count)."""
    return float(np.linalg.norm(W - U @ (U.T @ W), ord=2))
