"""Learned initial guesses for the periodic-orbit search (no counterpart in
the paper): a convolution network over r proposes a state correction, a
period T and an axial shift s from one snapshot; the recurrence scan of the
solver's own trajectories supplies the training labels and the plain
baseline guesses, and only the Newton residual certifies an orbit.

Features: the perturbation u - u_lam on the lowest modes |k| < 8, m < 8 --
3 components x 15 axial x 8 azimuthal x (re, im) = 720 channels at each of
the N radial points (layout [N][720], channel = ((c*15 + k)*8 + m)*2 + re/im).

Recurrence scan: for snapshots f_i (spacing dt_s)
D(i, tau) = min_s |sigma_s f_{i+tau} - f_i| / |f_i|, sigma_s the axial shift
(mode k times e^{i alpha k s}, the convention of the Newton residual
sigma_s Phi_T(u) - u).  As |sigma_s g - f|^2 = |f|^2 + |g|^2
- 2 Re sum_k c_k e^{i alpha k s} with c_k = <f_k, g_k>, all pairs come from one
Gram matrix per axial mode and the minimum over s is taken on a fine grid.

Labels: at a snapshot i whose best recurrence (T, s) has D < threshold the
network learns the closing correction (sigma_s f_{i+tau} - f_i) / 2 (the
midpoint of the two ends of the near-recurrence) and (T, cos 2 pi s/L,
sin 2 pi s/L).

Time integration runs in the library (opf_ens_*, opf_nk_solve), the network
in opf_net_*; this module arranges data and calls them.
"""
import math

import numpy as np

from . import inputs

KF, MF = 8, 8  # kept modes: |k| < KF, m < MF
NKF = 2 * KF - 1
NCH = 3 * NKF * MF * 2  # 720 channels
NOUT = 3  # T / T_scale, cos(2 pi s / L), sin(2 pi s / L)


def _check_modes(K, M):
    if K < KF or M < MF:
        raise ValueError(f"state needs |k| < {KF} and m < {MF} modes for the features")


def perturbation(U, K, N):
    """u - u_lam (Hagen-Poiseuille 1 - r^2 removed from the (0,0) u_z mode)."""
    V = np.array(U, dtype=np.complex128, copy=True)
    r = inputs.radial_points(N)
    V[2, 0, K - 1] -= 1.0 - r * r
    return V


def features(U, K, M, N):
    """Perturbation features [N][720] (float32) of a state (3, M, 2K-1, N)."""
    _check_modes(K, M)
    sub = perturbation(U, K, N)[:, :MF, K - KF:K + KF - 1]  # (3, MF, 15, N)
    sub = np.transpose(sub, (0, 2, 1, 3))  # (3, 15, MF, N)
    out = np.stack([sub.real, sub.imag], axis=3)  # (3, 15, MF, 2, N)
    return np.ascontiguousarray(out.reshape(NCH, N).T, dtype=np.float32)


def apply_features(U, delta, K, M, N):
    """U + delta on the kept modes (delta in the [N][720] feature layout)."""
    _check_modes(K, M)
    d = np.asarray(delta, dtype=np.float64).T.reshape(3, NKF, MF, 2, N)
    dc = np.transpose(d[:, :, :, 0] + 1j * d[:, :, :, 1], (0, 2, 1, 3))  # (3, MF, 15, N)
    V = np.array(U, dtype=np.complex128, copy=True)
    V[:, :MF, K - KF:K + KF - 1] += dc
    V[:, 0] = hermitian_m0(V[:, 0])  # a real field has A_{-k,0} = conj(A_{k,0})
    return V


def hermitian_m0(V0):
    """Project an m = 0 slice (3, 2K-1, N) onto A_{-k} = conj(A_k)."""
    return 0.5 * (V0 + np.conj(V0[:, ::-1]))


def shift_features(f, s, alpha):
    """sigma_s applied to features [..., N, 720]."""
    g = np.asarray(f, dtype=np.float64).reshape(f.shape[:-1] + (3, NKF, MF, 2))
    z = g[..., 0] + 1j * g[..., 1]
    k = np.arange(-(KF - 1), KF)
    z = z * np.exp(1j * alpha * k * s)[:, None]
    return np.stack([z.real, z.imag], axis=-1).reshape(f.shape)


def _complex_by_k(feats):
    """[S][N][720] -> complex [S][15][3*MF*N], grouped by axial mode."""
    S, N, _ = feats.shape
    f = np.asarray(feats, dtype=np.float64).reshape(S, N, 3, NKF, MF, 2)
    z = f[..., 0] + 1j * f[..., 1]  # (S, N, 3, 15, MF)
    z = np.transpose(z, (0, 3, 2, 4, 1))  # (S, 15, 3, MF, N)
    return z.reshape(S, NKF, -1)


def recurrence_matrix(feats, alpha, tau_min, tau_max, nshift=128):
    """D[i, tau - tau_min] and the minimising shift, for every pair in range
    (inf where i + tau runs past the end)."""
    z = _complex_by_k(feats)
    S = z.shape[0]
    nrm2 = (np.abs(z) ** 2).sum(axis=(1, 2))
    L = 2 * np.pi / alpha
    s_grid = np.arange(nshift) * L / nshift
    ph = np.exp(1j * alpha * np.outer(np.arange(-(KF - 1), KF), s_grid))  # (15, nshift)
    G = np.einsum("ikq,jkq->kij", np.conj(z), z, optimize=True)  # G[k, i, j] = <f_i,k, f_j,k>
    ntau = tau_max - tau_min + 1
    D = np.full((S, ntau), np.inf)
    Sh = np.zeros((S, ntau))
    for t in range(ntau):
        tau = tau_min + t
        if tau >= S:
            break
        i = np.arange(S - tau)
        c = G[:, i, i + tau].T  # (S - tau, 15)
        d2 = nrm2[i, None] + nrm2[i + tau, None] - 2.0 * np.real(c @ ph)
        j = np.argmin(d2, axis=1)
        D[i, t] = np.sqrt(np.maximum(d2[i, j], 0.0) / np.maximum(nrm2[i], 1e-300))
        Sh[i, t] = s_grid[j]
    return D, Sh


def best_recurrences(feats, alpha, dt_s, T_min, T_max, thresh=0.3, nshift=128, interior=True):
    """For each snapshot its best recurrence in [T_min, T_max]: list of
    (i, tau, T, s, D) with D < thresh.  interior: only dips of D in tau
    count (D[tau] no larger than at tau -+ 1, both inside the range), so a
    state that merely drifts slowly (D smallest at T_min) gives none."""
    tau_min = max(1, int(round(T_min / dt_s)))
    tau_max = int(round(T_max / dt_s))
    D, Sh = recurrence_matrix(feats, alpha, tau_min, tau_max, nshift)
    if interior:
        dip = np.zeros(D.shape, dtype=bool)
        dip[:, 1:-1] = (D[:, 1:-1] <= D[:, :-2]) & (D[:, 1:-1] <= D[:, 2:])
        D = np.where(dip, D, np.inf)
    t = np.argmin(D, axis=1)
    out = []
    for i in range(D.shape[0]):
        d = D[i, t[i]]
        if d < thresh:
            tau = tau_min + int(t[i])
            out.append((i, tau, tau * dt_s, float(Sh[i, t[i]]), float(d)))
    return out


def local_minima(recs):
    """Recurrences whose D is a local minimum along the trajectory."""
    byi = {r[0]: r for r in recs}
    out = []
    for r in recs:
        prv, nxt = byi.get(r[0] - 1), byi.get(r[0] + 1)
        if (prv is None or prv[4] >= r[4]) and (nxt is None or nxt[4] > r[4]):
            out.append(r)
    return out


def labels(feats, recs, alpha, T_scale):
    """(x, ty, tz) for the recurrences recs of one trajectory."""
    L = 2 * np.pi / alpha
    xs, tys, tzs = [], [], []
    for (i, tau, T, s, d) in recs:
        fi = feats[i].astype(np.float64)
        fe = shift_features(feats[i + tau], s, alpha)
        xs.append(fi)
        tys.append(0.5 * (fe - fi))
        tzs.append([T / T_scale, math.cos(2 * math.pi * s / L), math.sin(2 * math.pi * s / L)])
    return (np.asarray(xs, dtype=np.float32).reshape(-1, feats.shape[1], NCH),
            np.asarray(tys, dtype=np.float32).reshape(-1, feats.shape[1], NCH),
            np.asarray(tzs, dtype=np.float32).reshape(-1, NOUT))


def decode_z(z, alpha, T_scale):
    """Network head outputs -> (T, s in [0, L))."""
    L = 2 * np.pi / alpha
    z = np.asarray(z, dtype=np.float64)
    return z[:, 0] * T_scale, np.mod(np.arctan2(z[:, 2], z[:, 1]) * L / (2 * np.pi), L)


def constant_predictor_loss(ty, tz, lam, mean_tz, scale):
    """Training loss of the no-network guess (zero correction, the
    training-mean head), in the scaled units the network is trained in."""
    return float(np.mean((ty.astype(np.float64) / scale) ** 2) + lam * np.mean((tz - mean_tz[None]) ** 2))


# ---------------------------------------------------------------- GPU side


def generate(opf, N, K, M, m_p, alpha, Re, amp, seeds, dt, warmup, n_snap, every, keep=None,
             precision=1, rot=None):
    """Integrate one ensemble (trajectory j: Re[j], puff-envelope perturbation
    of amplitude amp[j] and seed seeds[j]) for `warmup` time units, then
    record features every `every` time units, n_snap times (fewer when keep
    is given: up to its largest index).  keep: {j: set of snapshot indices}
    whose full states are returned.  rot: frame rotation (Omega_x, Omega_y,
    Omega_z) shared by the trajectories (None: none).  Returns (feats
    [B][S][N][720], kept {(j, i): state}, finite [B] (False where a
    trajectory went non-finite), seconds)."""
    import time as _time

    B = len(Re)
    if keep is not None:
        n_snap = min(n_snap, 1 + max(max(v) for v in keep.values() if v))
    e = opf.opf_ens_create([N] * B, [K] * B, [M] * B, [m_p] * B, [alpha] * B, Re, [dt] * B)
    opf.opf_ens_set_option(e, "precision", precision)
    set_rotation(opf, e, rot)
    for j in range(B):
        opf.opf_ens_set_state(e, j, inputs.seeded_state(N, K, M, m_p, alpha, amp[j], seeds[j],
                                                        envelope=inputs.envelope_puff))
    feats = np.zeros((B, n_snap, N, NCH), dtype=np.float32)
    finite = np.ones(B, dtype=bool)
    kept = {}
    n_warm = int(round(warmup / dt))
    n_every = int(round(every / dt))
    t0 = _time.perf_counter()
    if n_warm:
        opf.opf_ens_step(e, n_warm)
    for i in range(n_snap):
        if i:
            opf.opf_ens_step(e, n_every)
        for j in range(B):
            if not finite[j]:
                continue
            U = opf.opf_ens_get_state(e, j)
            f = features(U, K, M, N)
            if not np.isfinite(f).all():
                finite[j] = False
                continue
            feats[j, i] = f
            if keep is not None and i in keep.get(j, ()):
                kept[(j, i)] = U
    seconds = _time.perf_counter() - t0
    opf.opf_ens_destroy(e)
    return feats, kept, finite, seconds


def rotate_features(f, a, phi, alpha, m_p):
    """Axial shift by a and azimuthal rotation by phi of features [B, N, 720]
    (one (a, phi) per sample): mode (k, m) times e^{i(alpha k a + m_p m phi)}.
    Both are symmetries of pipe flow; cylindrical components do not change
    under the rotation."""
    B, N, _ = f.shape
    g = f.reshape(B, N, 3, NKF, MF, 2).astype(np.float64)
    k = np.arange(-(KF - 1), KF)
    m = np.arange(MF)
    ph = np.exp(1j * (alpha * np.multiply.outer(a, k)[:, :, None] + m_p * np.multiply.outer(phi, m)[:, None, :]))
    z = (g[..., 0] + 1j * g[..., 1]) * ph[:, None, None, :, :]
    return np.stack([z.real, z.imag], axis=-1).reshape(f.shape).astype(np.float32)


def device_set(torch, data, scale):
    """The training set (x, ty, tz) resident on the device, features divided
    by scale (float32)."""
    x, ty, tz = data
    return (torch.from_numpy(np.ascontiguousarray(x / scale, dtype=np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(ty / scale, dtype=np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(tz, dtype=np.float32)).cuda())


def train(opf, torch, net, data, steps, batch, lr, lam, scale, seed=0, augment=None, dev=None):
    """Adam on minibatches of data = (x, ty, tz), features divided by scale.
    The set stays on the device (dev: a device_set of it, made here if
    None); each minibatch is gathered there by the library, and with
    augment = (alpha, m_p) each sample gets a random axial shift and
    azimuthal rotation (the labels T and s are invariant; the state
    correction turns with the state).  Returns the per-step losses."""
    x, ty, tz = data
    rng = np.random.default_rng(seed)
    dx, dy, dz = dev if dev is not None else device_set(torch, data, scale)
    rows, L = x.shape[0], x.shape[1]
    bx = torch.empty((batch,) + tuple(x.shape[1:]), dtype=torch.float32, device="cuda")
    by = torch.empty_like(bx)
    bz = torch.empty((batch, tz.shape[1]), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()  # the set and the buffers exist before the net's stream uses them
    losses = []
    for _ in range(steps):
        idx = rng.integers(0, rows, batch)
        ang = np.zeros((batch, 2))
        if augment is not None:
            al, mp = augment
            ang[:, 0] = al * rng.uniform(0.0, 2 * np.pi / al, batch)   # alpha a
            ang[:, 1] = mp * rng.uniform(0.0, 2 * np.pi / mp, batch)   # m_p phi
        opf.opf_net_gather_augment(net, dx.data_ptr(), dy.data_ptr(), dz.data_ptr(), rows, idx, ang, L, 3, NKF, MF,
                                   tz.shape[1], bx.data_ptr(), by.data_ptr(), bz.data_ptr())
        losses.append(opf.opf_net_train_step(net, bx.data_ptr(), by.data_ptr(), bz.data_ptr(), batch, lam, lr))
    return losses


def evaluate_loss(opf, torch, net, data, lam, scale):
    """Loss of the network on data (in the scaled units used for training)."""
    x, ty, tz = data
    y, z = forward(opf, torch, net, x, scale)
    return float(np.mean(((y - ty) / scale) ** 2) + lam * np.mean((z - tz) ** 2))


def forward(opf, torch, net, feats, scale):
    """Network outputs for feature arrays [B][N][720]: (corrections, head)."""
    B = feats.shape[0]
    dx = torch.from_numpy(np.ascontiguousarray(feats / scale, dtype=np.float32)).cuda()
    dy = torch.empty_like(dx)
    dz = torch.empty((B, NOUT), dtype=torch.float32, device="cuda")
    opf.opf_net_forward(net, dx.data_ptr(), B, dy.data_ptr(), dz.data_ptr())
    torch.cuda.synchronize()
    return dy.cpu().numpy().astype(np.float64) * scale, dz.cpu().numpy().astype(np.float64)


def shifted(U, s, alpha, K):
    """sigma_s U for a full state (3, M, 2K-1, N)."""
    k = np.arange(-(K - 1), K)
    return U * np.exp(1j * alpha * k * s)[None, None, :, None]


def packed_norm(U, K):
    """Norm over the independent coefficients (m = 0 with k >= 0, all k for
    m > 0): the normalisation opf_nk_solve reports its residual in."""
    w = np.ones(U.shape[1:3])
    w[0, :K - 1] = 0.0
    return float(np.sqrt((w[None, :, :, None] * np.abs(U) ** 2).sum()))


def set_rotation(opf, e, rot):
    """Frame rotation (Omega_x, Omega_y, Omega_z) of every trajectory of ensemble e."""
    if rot is not None:
        for key, v in zip(("rot_x", "rot_y", "rot_z"), rot):
            opf.opf_ens_set_option(e, key, float(v))


def relative_residual(opf, N, K, M, m_p, alpha, Re, states, T, s, dt, rot=None):
    """|sigma_s Phi_T(u) - u| / |u| (packed norms) for a list of guesses,
    batched in one ensemble; all take the same number of steps,
    ceil(max T / dt), each of its own length T_j / steps."""
    B = len(states)
    nmax = max(max(1, int(math.ceil(t / dt - 1e-9))) for t in T)
    e = opf.opf_ens_create([N] * B, [K] * B, [M] * B, [m_p] * B, [alpha] * B, Re, [t / nmax for t in T])
    set_rotation(opf, e, rot)
    for j in range(B):
        opf.opf_ens_set_state(e, j, states[j])
    opf.opf_ens_step(e, nmax)
    out = np.empty(B)
    for j in range(B):
        V = shifted(opf.opf_ens_get_state(e, j), s[j], alpha, K)
        out[j] = packed_norm(V - states[j], K) / packed_norm(states[j], K)
    opf.opf_ens_destroy(e)
    return out


def run_pipeline(opf, torch, cfg, log=None):
    """Snapshots -> recurrence labels -> training -> Newton-Krylov on held-out
    recurrences with and without the network.  Returns a dict of measurements
    (losses, timings, per-arm Newton results).  cfg keys: N K M m_p alpha dt
    precision Re_train Re_test amp B_train B_test seed warmup n_snap every
    T_min T_max thresh hidden steps batch lr lam net_seed nk_guesses nk_T_max
    nk (options of opf_nk_solve); optional B_val eval_every augment
    interior_minima rot (frame rotation (Omega_x, Omega_y, Omega_z) of the
    data and of the Newton problems)."""
    import time as _time

    say = log or (lambda *a: None)
    c = dict(cfg)
    N, K, M, m_p, alpha = c["N"], c["K"], c["M"], c["m_p"], c["alpha"]
    Btr, Bte = c["B_train"], c["B_test"]
    rng = np.random.default_rng(c["seed"])
    Re = list(rng.uniform(c["Re_train"][0], c["Re_train"][1], Btr)) + [float(c["Re_test"])] * Bte
    lo, hi = np.log(c["amp"][0]), np.log(c["amp"][1])
    amp = list(np.exp(rng.uniform(lo, hi, Btr + Bte)))
    seeds = [int(c["seed"]) * 1000 + j for j in range(Btr + Bte)]
    out = {"config": {k: v for k, v in c.items() if k != "nk"}, "nk_options": dict(c.get("nk", {}))}

    rot = c.get("rot")
    feats, _, finite, t_gen = generate(opf, N, K, M, m_p, alpha, Re, amp, seeds, c["dt"], c["warmup"],
                                       c["n_snap"], c["every"], precision=c.get("precision", 1), rot=rot)
    steps_per_traj = int(round(c["warmup"] / c["dt"])) + (c["n_snap"] - 1) * int(round(c["every"] / c["dt"]))
    out["generate"] = {"seconds": t_gen, "trajectories": Btr + Bte, "finite": int(finite.sum()),
                       "snapshots": int(finite.sum()) * c["n_snap"],
                       "trajectory_steps_per_s": (Btr + Bte) * steps_per_traj / t_gen}
    say("generate", out["generate"])

    t0 = _time.perf_counter()
    recs = [best_recurrences(feats[j], alpha, c["every"], c["T_min"], c["T_max"], c["thresh"],
                             interior=c.get("interior_minima", True))
            if finite[j] else [] for j in range(Btr + Bte)]
    out["scan_seconds"] = _time.perf_counter() - t0
    T_scale = float(c["T_max"])

    def gather(js):
        parts = [labels(feats[j], recs[j], alpha, T_scale) for j in js if recs[j]]
        if not parts:
            return None
        return tuple(np.concatenate([p[q] for p in parts]) for q in range(3))

    Bval = int(c.get("B_val", max(1, Btr // 8)))
    train_set = gather(range(Btr - Bval))
    val_set = gather(range(Btr - Bval, Btr))
    test_set = gather(range(Btr, Btr + Bte))
    count = lambda d: 0 if d is None else int(d[0].shape[0])
    out["samples"] = {"train": count(train_set), "validation": count(val_set), "test": count(test_set)}
    say("samples", out["samples"])
    if train_set is None or test_set is None or val_set is None:
        return out

    scale = float(np.sqrt(np.mean(train_set[0].astype(np.float64) ** 2)))
    mean_tz = train_set[2].astype(np.float64).mean(axis=0)
    net = opf.opf_net_create(NCH, c["hidden"], N, NOUT, seed=c["net_seed"])
    out["params"] = int(opf.opf_net_param_count(net)[0])
    # start from the no-network guess: zero correction, training-mean head
    p, sizes = opf.opf_net_get_params(net), opf.opf_net_param_count(net)[1]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    p[offs[4]:offs[6]] = 0.0  # W3, b3
    p[offs[6]:offs[7]] = 0.0  # Wh
    p[offs[7]:offs[8]] = mean_tz  # bh
    opf.opf_net_set_params(net, p)
    lam = c["lam"]
    every = int(c.get("eval_every", 100))
    best = (evaluate_loss(opf, torch, net, val_set, lam, scale), 0, p.copy())
    losses = []
    torch.cuda.synchronize()
    t0 = _time.perf_counter()
    dev = device_set(torch, train_set, scale)
    for r in range(0, c["steps"], every):
        losses += train(opf, torch, net, train_set, min(every, c["steps"] - r), c["batch"], c["lr"], lam, scale,
                        seed=c["seed"] + r, augment=(alpha, m_p) if c.get("augment", True) else None, dev=dev)
        v = evaluate_loss(opf, torch, net, val_set, lam, scale)
        if v < best[0]:
            best = (v, r + every, opf.opf_net_get_params(net))
    torch.cuda.synchronize()
    t_train = _time.perf_counter() - t0
    opf.opf_net_set_params(net, best[2])  # early stopping on the validation trajectories
    out["train"] = {"seconds": t_train, "steps": c["steps"], "batch": c["batch"], "best_step": best[1],
                    "validation_loss": best[0],
                    "loss_first": float(np.mean(losses[:10])), "loss_last": float(np.mean(losses[-10:]))}
    out["loss"] = {
        "train_net": evaluate_loss(opf, torch, net, train_set, lam, scale),
        "train_const": constant_predictor_loss(train_set[1], train_set[2], lam, mean_tz, scale),
        "test_net": evaluate_loss(opf, torch, net, test_set, lam, scale),
        "test_const": constant_predictor_loss(test_set[1], test_set[2], lam, mean_tz, scale)}
    _, zt = forward(opf, torch, net, test_set[0], scale)
    Tn, _ = decode_z(zt, alpha, T_scale)
    Tt, _ = decode_z(test_set[2], alpha, T_scale)
    out["T_abs_err_test"] = {"net": float(np.mean(np.abs(Tn - Tt))),
                             "const": float(np.mean(np.abs(mean_tz[0] * T_scale - Tt)))}
    say("loss", out["loss"], out["T_abs_err_test"])

    # held-out Newton-Krylov starts: the best local minima of the scan
    cands = sorted((r[4], j, r) for j in range(Btr, Btr + Bte)
                   for r in local_minima(recs[j]) if r[2] <= c["nk_T_max"])[:c["nk_guesses"]]
    out["nk_starts"] = [(int(j), int(r[0]), float(r[2]), float(r[3]), float(r[4])) for _, j, r in cands]
    if not cands:
        return out
    keep = {}
    for _, j, r in cands:
        keep.setdefault(j - Btr, set()).add(r[0])
    feats2, kept, _, _ = generate(opf, N, K, M, m_p, alpha, Re[Btr:], amp[Btr:], seeds[Btr:], c["dt"],
                                  c["warmup"], c["n_snap"], c["every"], keep=keep,
                                  precision=c.get("precision", 1), rot=rot)
    out["replay_max_abs_diff"] = float(max(np.abs(feats2[j - Btr, r[0]] - feats[j, r[0]]).max()
                                           for _, j, r in cands))
    U0 = [kept[(j - Btr, r[0])] for _, j, r in cands]
    T_rec = [r[2] for _, _, r in cands]
    s_rec = [r[3] for _, _, r in cands]
    y, z = forward(opf, torch, net, np.stack([features(u, K, M, N) for u in U0]), scale)
    T_net, s_net = decode_z(z, alpha, T_scale)
    T_net = np.clip(T_net, c["T_min"], c["T_max"])
    U_net = [apply_features(u, y[q], K, M, N) for q, u in enumerate(U0)]
    T_mean, s_mean = decode_z(mean_tz[None, :], alpha, T_scale)
    T_mean = float(np.clip(T_mean[0], c["T_min"], c["T_max"]))
    arms = {"recurrence": (U0, T_rec, s_rec),
            "learned": (U_net, list(T_net), list(s_net)),
            "learned_state_recurrence_T": (U_net, T_rec, s_rec),
            # the single-snapshot guess without a network: the snapshot with the
            # training-mean period and shift
            "snapshot_mean_T": (U0, [T_mean] * len(U0), [float(s_mean[0])] * len(U0))}
    nk = dict(c.get("nk", {}))
    if rot is not None:
        nk.setdefault("rot", tuple(float(v) for v in rot))
    Re_te = [float(c["Re_test"])] * len(U0)
    out["nk"] = {}
    for name, (Us, Ts, ss) in arms.items():
        r0 = relative_residual(opf, N, K, M, m_p, alpha, Re_te, Us, Ts, ss, nk.get("dt", 0.01), rot=rot)
        t0 = _time.perf_counter()
        st, T, s, res, it = opf.opf_nk_solve(N, K, M, m_p, alpha, float(c["Re_test"]), Us, Ts, ss, **nk)
        sec = _time.perf_counter() - t0
        tol = nk.get("tol", 1e-10)
        ok = np.asarray(res) < tol
        its = np.asarray(it)
        out["nk"][name] = {"initial_residual": [float(v) for v in r0], "final_residual": [float(v) for v in res],
                           "newton_iterations": [int(v) for v in it], "T": [float(v) for v in T],
                           "s": [float(v) for v in s],
                           "converged": int(ok.sum()), "guesses": len(Us), "seconds": sec,
                           "certified_fraction": float(ok.mean()),
                           # the guesses of an arm are solved together (one batched solve),
                           # so the time to certification is given in Newton iterations
                           "median_newton_iterations_to_certification": float(np.median(its[ok])) if ok.any() else None,
                           "median_initial": float(np.median(r0)), "median_final": float(np.median(res))}
        say("nk", name, {k: out["nk"][name][k] for k in ("median_initial", "median_final", "converged", "seconds")})
    opf.opf_net_destroy(net)
    return out
