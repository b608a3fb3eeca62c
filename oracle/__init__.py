"""FP64 CPU oracle for the EPSR hot path -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference arms of
`bench.py` may import this package. The CUDA library and its binding never do; they
share no code, header, table or constant with it.

The C part (`epsr_oracle.c`) holds the pair loops (minimum image, exact integer
squared distances, bins, energies, moves, histograms, Eq. (1), smeared histograms and
their adjoint). This module wraps it with ctypes and adds the small dense pieces in
NumPy: the Eq. (1) weight factors, the Poisson empirical-potential basis and its
closed-form Q-space transform, the least-squares fit of the basis to a Delta S(Q),
and the chi^2 of the differentiable form. Citations are to NeuDATool
(arXiv:1904.08756): sections, equations, and the readings where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epsr_oracle.c")
_LIB = os.path.join(_HERE, "libepsr_oracle.so")
MAX_TYPES = 8
MAX_MOL_ATOMS = 64


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -ffp-contract=off so that FP64 sequences are exact)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "epsr_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcSystem(C.Structure):
    _fields_ = [("n_atoms", C.c_int64), ("n_mol", C.c_int64), ("L_fx", C.c_int64),
                ("n_types", C.c_int32), ("scale_log2", C.c_int32),
                ("xyz", C.POINTER(C.c_int32)), ("type", C.POINTER(C.c_int32)),
                ("mol_start", C.POINTER(C.c_int64)),
                ("q", C.c_double * MAX_TYPES), ("sigma", C.c_double * MAX_TYPES),
                ("eps", C.c_double * MAX_TYPES), ("r_coul", C.c_double),
                ("bin_p", C.c_int32), ("bin_q", C.c_int32), ("n_bins", C.c_int32),
                ("rigid", C.c_int32), ("flexible", C.c_int32),
                ("bond_k", C.c_double * (MAX_TYPES * MAX_TYPES)),
                ("bond_d", C.c_double * (MAX_TYPES * MAX_TYPES)), ("temperature", C.c_double),
                ("max_translation", C.c_double), ("max_rotation_deg", C.c_double),
                ("ep", C.POINTER(C.c_double)), ("r_lj", C.c_double)]


class OrcStats(C.Structure):
    _fields_ = [("attempted", C.c_int64), ("accepted", C.c_int64), ("sum_dU", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        sysp = P(OrcSystem)
        L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.orc_coulomb_constant.restype = C.c_double
        L.orc_gas_constant.restype = C.c_double
        L.orc_min_image.argtypes = [C.c_int64, C.c_int64]
        L.orc_min_image.restype = C.c_int64
        L.orc_dist2_points.argtypes = [P(C.c_int32), P(C.c_int32), C.c_int64]
        L.orc_dist2_points.restype = C.c_int64
        L.orc_bin_index.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int32]
        L.orc_bin_index.restype = C.c_int64
        L.orc_pair_index.argtypes = [C.c_int32, C.c_int32, C.c_int32]
        L.orc_pair_index.restype = C.c_int32
        L.orc_pair_energy.argtypes = [sysp, C.c_int32, C.c_int32, C.c_int64]
        L.orc_pair_energy.restype = C.c_double
        L.orc_total_energy.argtypes = [sysp]
        L.orc_total_energy.restype = C.c_double
        L.orc_propose.argtypes = [sysp, C.c_uint64, C.c_uint64, C.c_uint32, P(C.c_int64),
                                  P(C.c_int32), P(C.c_double)]
        L.orc_delta_u.argtypes = [sysp, C.c_int64, P(C.c_int32), P(C.c_double)]
        L.orc_delta_u.restype = C.c_double
        L.orc_accept.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_accept.restype = C.c_int
        L.orc_mc_sweep.argtypes = [sysp, C.c_int64, C.c_uint64, C.c_uint64, C.c_uint32,
                                   P(OrcStats)]
        L.orc_histogram.argtypes = [sysp, C.c_int64, C.c_int64, P(C.c_uint64)]
        L.orc_histogram_omp.argtypes = [sysp, P(C.c_uint64), C.c_int]
        L.orc_normalize_g.argtypes = [sysp, P(C.c_uint64), C.c_int64, P(C.c_double)]
        L.orc_sq.argtypes = [P(C.c_double), C.c_int32, C.c_int32, C.c_double, P(C.c_double),
                             C.c_int32, P(C.c_double), C.c_int32, P(C.c_double),
                             P(C.c_double), P(C.c_double)]
        L.orc_smeared_hist.argtypes = [sysp, C.c_double, P(C.c_double)]
        L.orc_smeared_grad.argtypes = [sysp, C.c_double, P(C.c_double), P(C.c_double)]
        L.orc_smeared_grad_atoms.argtypes = [sysp, C.c_double, P(C.c_double), P(C.c_int64),
                                             C.c_int64, P(C.c_double)]
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ------------------------------------------------------------------------------------
# Box wrapper
# ------------------------------------------------------------------------------------

class Box:
    """Oracle view of a System (owns copies of the arrays; xyz is updated by MC)."""

    def __init__(self, system, xyz: np.ndarray | None = None, ep: np.ndarray | None = None):
        self.sys = system
        self.xyz = np.ascontiguousarray(system.xyz if xyz is None else xyz, np.int32).copy()
        self.type = np.ascontiguousarray(system.type, np.int32)
        self.mol_start = np.ascontiguousarray(system.mol_start, np.int64)
        self.ep = None if ep is None else np.ascontiguousarray(ep, np.float64)
        st = OrcSystem()
        st.n_atoms = system.n_atoms
        st.n_mol = system.n_mol
        st.L_fx = system.L_fx
        st.n_types = system.n_types
        st.scale_log2 = 20
        st.xyz = _ptr(self.xyz, C.c_int32)
        st.type = _ptr(self.type, C.c_int32)
        st.mol_start = _ptr(self.mol_start, C.c_int64)
        for i in range(system.n_types):
            st.q[i] = system.q[i]
            st.sigma[i] = system.sigma[i]
            st.eps[i] = system.eps[i]
        st.r_coul = system.r_coul
        st.bin_p, st.bin_q, st.n_bins = system.bin_p, system.bin_q, system.n_bins
        st.rigid = 1 if system.rigid_molecules else 0
        st.flexible = 1 if getattr(system, "flexible", False) else 0
        if st.flexible:
            for a in range(system.n_types):
                for b in range(system.n_types):
                    st.bond_k[a * MAX_TYPES + b] = float(system.bond_k[a][b])
                    st.bond_d[a * MAX_TYPES + b] = float(system.bond_d[a][b])
        st.temperature = system.temperature
        st.max_translation = system.max_translation
        st.max_rotation_deg = system.max_rotation_deg
        st.ep = _ptr(self.ep, C.c_double) if self.ep is not None else C.POINTER(C.c_double)()
        st.r_lj = float(getattr(system, "r_lj", 0.0))
        self.st = st

    @property
    def n_pairs(self) -> int:
        t = self.sys.n_types
        return t * (t + 1) // 2

    def ref(self):
        return C.byref(self.st)

    # --- energies and moves --------------------------------------------------------
    def pair_energy(self, ta: int, tb: int, d2: int) -> float:
        return lib().orc_pair_energy(self.ref(), ta, tb, int(d2))

    def total_energy(self) -> float:
        return lib().orc_total_energy(self.ref())

    def propose(self, seed: int, move: int, box_index: int = 0):
        mol = C.c_int64()
        u = C.c_double()
        trial = np.zeros((MAX_MOL_ATOMS, 3), np.int32)
        lib().orc_propose(self.ref(), seed, move, box_index, C.byref(mol),
                          _ptr(trial, C.c_int32), C.byref(u))
        m = int(self.mol_start[mol.value + 1] - self.mol_start[mol.value])
        return mol.value, trial[:m].copy(), u.value

    def delta_u(self, mol: int, trial: np.ndarray):
        t = np.ascontiguousarray(trial, np.int32)
        cond = C.c_double()
        dU = lib().orc_delta_u(self.ref(), mol, _ptr(t, C.c_int32), C.byref(cond))
        return dU, cond.value

    def apply(self, mol: int, trial: np.ndarray):
        a0, a1 = int(self.mol_start[mol]), int(self.mol_start[mol + 1])
        self.xyz[a0:a1] = trial

    def mc_sweep(self, n_moves: int, seed: int, move0: int = 0, box_index: int = 0):
        st = OrcStats()
        lib().orc_mc_sweep(self.ref(), n_moves, seed, move0, box_index, C.byref(st))
        return st.attempted, st.accepted, st.sum_dU

    def set_ep(self, ep):
        """Replaces the empirical-potential table (FP64 [n_pairs][n_bins], or None for zero)."""
        self.ep = None if ep is None else np.ascontiguousarray(ep, np.float64)
        self.st.ep = _ptr(self.ep, C.c_double) if self.ep is not None else C.POINTER(C.c_double)()

    # --- histograms and g(r) --------------------------------------------------------
    def histogram(self, i0: int = 0, i1: int | None = None, threads: int = 1) -> np.ndarray:
        H = np.zeros((self.n_pairs, self.sys.n_bins), np.uint64)
        if threads == 1 or i0 != 0 or i1 is not None:
            lib().orc_histogram(self.ref(), i0, self.sys.n_atoms if i1 is None else i1,
                                _ptr(H, C.c_uint64))
        else:
            lib().orc_histogram_omp(self.ref(), _ptr(H, C.c_uint64), threads)
        return H

    def normalize_g(self, H: np.ndarray, n_configs: int = 1) -> np.ndarray:
        H = np.ascontiguousarray(H, np.uint64)
        g = np.zeros(H.shape, np.float64)
        lib().orc_normalize_g(self.ref(), _ptr(H, C.c_uint64), n_configs, _ptr(g, C.c_double))
        return g

    def smeared_hist(self, sigma: float) -> np.ndarray:
        Ht = np.zeros((self.n_pairs, self.sys.n_bins), np.float64)
        lib().orc_smeared_hist(self.ref(), sigma, _ptr(Ht, C.c_double))
        return Ht

    def smeared_grad(self, sigma: float, lam: np.ndarray, atoms: np.ndarray | None = None):
        lam = np.ascontiguousarray(lam, np.float64)
        if atoms is None:
            g = np.zeros((self.sys.n_atoms, 3), np.float64)
            lib().orc_smeared_grad(self.ref(), sigma, _ptr(lam, C.c_double), _ptr(g, C.c_double))
            return g
        idx = np.ascontiguousarray(atoms, np.int64)
        g = np.zeros((len(idx), 3), np.float64)
        lib().orc_smeared_grad_atoms(self.ref(), sigma, _ptr(lam, C.c_double),
                                     _ptr(idx, C.c_int64), len(idx), _ptr(g, C.c_double))
        return g


# ------------------------------------------------------------------------------------
# Scalar helpers
# ------------------------------------------------------------------------------------

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def coulomb_constant() -> float:
    return lib().orc_coulomb_constant()


def gas_constant() -> float:
    return lib().orc_gas_constant()


def min_image(dx: int, L: int) -> int:
    return lib().orc_min_image(int(dx), int(L))


def bin_index(d2: int, p: int, q: int, scale_log2: int = 20) -> int:
    return lib().orc_bin_index(int(d2), p, q, scale_log2)


def pair_index(a: int, b: int, n_types: int) -> int:
    return lib().orc_pair_index(a, b, n_types)


def accept(dU: float, u_acc: float, temperature: float) -> bool:
    return bool(lib().orc_accept(dU, u_acc, temperature))


# ------------------------------------------------------------------------------------
# Eq. (1): weights and the sine transform
# ------------------------------------------------------------------------------------

def concentrations(system) -> np.ndarray:
    counts = np.bincount(system.type, minlength=system.n_types).astype(np.float64)
    return counts / counts.sum()


def eq1_weights(system):
    """Per pair (a <= b): (2 - delta_ab) c_a c_b b_a b_b, and the flat background
    sum_a c_a b_a^2 (Eq. 1). b in units of 1e-12 cm (fm / 10) so S(Q) is in barn."""
    c = concentrations(system)
    b = np.asarray(system.b, np.float64) / 10.0
    T = system.n_types
    W = np.zeros(T * (T + 1) // 2)
    for a in range(T):
        for bb in range(a, T):
            W[pair_index(a, bb, T)] = (1.0 if a == bb else 2.0) * c[a] * c[bb] * b[a] * b[bb]
    flat = float((c * b * b).sum())
    return W, flat


def number_density(system) -> float:
    return system.n_atoms / system.L ** 3


def sq(g: np.ndarray, dr: float, Q: np.ndarray, w: np.ndarray, cols_per_set: int,
       flat: np.ndarray):
    """Eq. (1) for columns g [n_cols][n_bins] -> (S_partial [n_cols][nQ], S_total)."""
    g = np.ascontiguousarray(g, np.float64)
    Q = np.ascontiguousarray(Q, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    flat = np.ascontiguousarray(np.atleast_1d(flat), np.float64)
    n_cols, n_bins = g.shape
    Sp = np.zeros((n_cols, len(Q)))
    St = np.zeros((n_cols // cols_per_set, len(Q)))
    lib().orc_sq(_ptr(g, C.c_double), n_cols, n_bins, dr, _ptr(Q, C.c_double), len(Q),
                 _ptr(w, C.c_double), cols_per_set, _ptr(flat, C.c_double),
                 _ptr(Sp, C.c_double), _ptr(St, C.c_double))
    return Sp, St


def sq_of_box(box: Box, g: np.ndarray, Q: np.ndarray | None = None):
    """S(Q) of one box from its g_ab(r) (Eq. 1) -> (S_partial, S_total[nQ])."""
    s = box.sys
    W, flat = eq1_weights(s)
    rho = number_density(s)
    Q = s.Q if Q is None else Q
    Sp, St = sq(g, s.dr, Q, 4.0 * math.pi * rho * W, len(W), np.array([flat]))
    return Sp, St[0]


# ------------------------------------------------------------------------------------
# Empirical potential: Poisson basis (Sec. 2.1, Fig. 1) and the fit of Delta S(Q)
# ------------------------------------------------------------------------------------

def poisson_p(n: int, s: float, r: np.ndarray) -> np.ndarray:
    """p_n(r) = (r / (n s))^n exp(n - r / s): a Poisson-shaped function of r with its
    peak, of height 1, at r = n s (Fig. 1: peaks normalised to 1; reading c14)."""
    r = np.asarray(r, np.float64)
    with np.errstate(divide="ignore"):
        return np.exp(n * np.log(np.where(r > 0, r, 1.0) / (n * s)) + n - r / s) * (r > 0)


def poisson_F(n: int, s: float, Q: np.ndarray, rho: float) -> np.ndarray:
    """4 pi rho int_0^inf r^2 p_n(r) sin(Qr)/(Qr) dr in closed form (reading c14):
    (4 pi rho / Q) e^n / (n s)^n Gamma(n+2) s^(n+2) sin((n+2) atan(Q s)) / (1+Q^2 s^2)^((n+2)/2)
    from int_0^inf r^m e^(-r/s) sin(Qr) dr = Gamma(m+1) Im[(1/s - iQ)^-(m+1)]."""
    Q = np.asarray(Q, np.float64)
    m = n + 2
    logc = n - n * math.log(n * s) + math.lgamma(m) + m * math.log(s)
    return (4.0 * math.pi * rho / Q) * np.exp(logc - 0.5 * m * np.log1p((Q * s) ** 2)) \
        * np.sin(m * np.arctan(Q * s))


def ep_basis_matrix(n_basis: int, s: float, Q: np.ndarray, rho: float) -> np.ndarray:
    """F [nQ][n_basis] with F[:, n-1] = poisson_F(n, ...)."""
    return np.stack([poisson_F(n, s, Q, rho) for n in range(1, n_basis + 1)], axis=1)


def pair_resolve(dS: np.ndarray, w: np.ndarray, gamma: float = 0.0) -> np.ndarray:
    """Pair-resolved Delta S_p from per-dataset Delta S_i = sum_p w_ip Delta S_p (Eq. 2
    uses the inverse of the weight matrix; for fewer datasets than pairs the matrix is
    stacked on gamma * I and pseudo-inverted, reading c16). dS [n_data][nQ], w [n_data][P]."""
    w = np.asarray(w, np.float64)
    n_data, P = w.shape
    A = np.vstack([w, gamma * np.eye(P)]) if gamma > 0 else w
    rhs = np.vstack([dS, np.zeros((P, dS.shape[1]))]) if gamma > 0 else dS
    return np.linalg.pinv(A) @ rhs


def ep_fit(dSp: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Least-squares coefficients C [P][n_basis] with dSp[p] ~ F @ C[p] (Sec. 2.1:
    the Q-space Poisson series is fitted to Delta S(Q))."""
    C_, *_ = np.linalg.lstsq(F, np.asarray(dSp, np.float64).T, rcond=None)
    return C_.T


def ep_table(C_: np.ndarray, s: float, n_bins: int, dr: float, alpha: float, kT: float):
    """U_EP[p][k] = -alpha kT sum_n C[p][n] p_n(r_k), r_k = (k + 1/2) dr (reading c13)."""
    r = (np.arange(n_bins) + 0.5) * dr
    Pm = np.stack([poisson_p(n, s, r) for n in range(1, C_.shape[1] + 1)], axis=0)
    return -alpha * kT * (C_ @ Pm)


# ------------------------------------------------------------------------------------
# Differentiable form: chi^2 of the smeared S(Q) and its adjoint pieces
# ------------------------------------------------------------------------------------

def smeared_g(box: Box, Ht: np.ndarray) -> np.ndarray:
    """g~ from the smeared counts, normalised as g (reading c7): same factors as
    orc_normalize_g applied to real-valued counts."""
    s = box.sys
    dr = s.dr
    V = s.L ** 3
    counts = np.bincount(s.type, minlength=s.n_types).astype(np.float64)
    k = np.arange(s.n_bins)
    shell = 4.0 * math.pi / 3.0 * (((k + 1) * dr) ** 3 - (k * dr) ** 3)
    g = np.zeros_like(Ht)
    for a in range(s.n_types):
        for b in range(a, s.n_types):
            p = pair_index(a, b, s.n_types)
            Pab = 0.5 * counts[a] * (counts[a] - 1) if a == b else counts[a] * counts[b]
            g[p] = Ht[p] * V / (Pab * shell)
    return g, V / (np.array([0.5 * counts[a] * (counts[a] - 1) if a == b else counts[a] * counts[b]
                             for a in range(s.n_types) for b in range(a, s.n_types)])[:, None]
                    * shell[None, :])


def sine_matrix(Q: np.ndarray, n_bins: int, dr: float) -> np.ndarray:
    """K[i, k] = r_k^2 dr sin(Q_i r_k) / (Q_i r_k), r_k = (k + 1/2) dr (Eq. 1, midpoint)."""
    r = (np.arange(n_bins) + 0.5) * dr
    x = np.outer(Q, r)
    return (r * r * dr)[None, :] * np.sin(x) / x


def chi2_and_grads(box: Box, sigma: float, Q: np.ndarray, target: np.ndarray,
                   C_: np.ndarray, s_basis: float, grad_atoms: np.ndarray | None = None):
    """chi^2(x, C) = sum_Q [S~(Q; x) + sum_p W_p sum_n C_pn F_n(Q) - T(Q)]^2 (reading
    c15), with S~ the Eq. (1) transform of the smeared g~ (orc_sq, the routine that gives
    S(Q) of an exact histogram; sine_matrix is the K of that sum, used by the adjoint).
    Returns chi^2, dchi2/dC [P][n_basis], dchi2/dx [n_atoms or len(grad_atoms)][3] (per
    Angstrom), S~ and lambda = dchi2/dHt."""
    s = box.sys
    W, flat = eq1_weights(s)
    rho = number_density(s)
    Ht = box.smeared_hist(sigma)
    g, fac = smeared_g(box, Ht)
    K = sine_matrix(Q, s.n_bins, s.dr)
    wcol = 4.0 * math.pi * rho * W
    _, St = sq(g, s.dr, Q, wcol, len(W), np.array([flat]))   # Eq. (1) through orc_sq
    S_t = St[0]
    F = ep_basis_matrix(C_.shape[1], s_basis, Q, rho)     # [nQ][n_basis]
    ep_img = (W[:, None] * (C_ @ F.T)).sum(axis=0)
    res = S_t + ep_img - target
    chi2 = float((res * res).sum())
    dC = 2.0 * W[:, None] * (F.T @ res)[None, :]          # [P][n_basis]
    lam = (2.0 * wcol[:, None] * (res @ K)[None, :]) * fac  # dchi2/dHt [P][n_bins]
    if grad_atoms is None:
        gx = box.smeared_grad(sigma, lam)
    else:
        gx = box.smeared_grad(sigma, lam, grad_atoms)
    return chi2, dC, gx, S_t, lam


# ------------------------------------------------------------------------------------
# The refinement loop (Sec. 2.2 items III-VI; Sec. 2.1; Eq. 2)
# ------------------------------------------------------------------------------------

def refine_pass(ob: Box, target: np.ndarray, w: np.ndarray, flat: np.ndarray, Q: np.ndarray,
                n_basis: int, s_basis: float, gamma: float, alpha: float,
                H_acc: np.ndarray | None = None, n_cfg: int = 0,
                moves: int = 0, seed: int = 0, move0: int = 0):
    """One pass of the loop, in the paper's order:
      III  `moves` Metropolis moves of the oracle's chain (none when the caller has already
           moved the box, e.g. by replaying another implementation's decisions);
      VI   the pair histogram of this configuration added to H_acc (n_cfg configurations so
           far; H_acc None starts afresh) and g_ab from the accumulated counts;
      IV   S_d(Q) of every dataset d by Eq. (1) with the dataset's weights w[d] (barn,
           without 4 pi rho) and background flat[d]; Delta S_d = target_d - S_d, chi^2;
      V    the pair-resolved Delta S_p (pseudo-inverse of the weights, reading c16), its
           least-squares Poisson coefficients C (Sec. 2.1) and the table update
           -alpha kT sum_n C_pn p_n(r_k) (reading c13) added to the box's EP table.
    Returns a dict with H, n_cfg, g, S, dS, chi2, C and the new table."""
    s = ob.sys
    if moves:
        ob.mc_sweep(moves, seed, move0)
    H = ob.histogram()
    H = H if H_acc is None else H_acc + H
    n_cfg = 1 if H_acc is None else n_cfg + 1
    g = ob.normalize_g(H, n_cfg)
    w = np.asarray(w, np.float64)
    n_data, P = w.shape
    rho = number_density(s)
    _, S = sq(np.tile(g, (n_data, 1)), s.dr, Q, (4.0 * math.pi * rho * w).ravel(), P,
              np.asarray(flat, np.float64))
    dS = np.asarray(target, np.float64) - S
    chi2 = float((dS * dS).sum())
    dSp = pair_resolve(dS, w, gamma)
    C_ = ep_fit(dSp, ep_basis_matrix(n_basis, s_basis, Q, rho))
    kT = gas_constant() * s.temperature
    table = ep_table(C_, s_basis, s.n_bins, s.dr, alpha, kT)
    ep = table if ob.ep is None else ob.ep + table
    ob.set_ep(ep)
    return {"H": H, "n_cfg": n_cfg, "g": g, "S": S, "dS": dS, "chi2": chi2, "C": C_, "ep": ep}
