"""Seeded synthetic crystals with time-reversal-symmetric Bloch states.

Everything here is input preparation (what a ground-state code would
provide).  Conventions:

* Hartree atomic units: energies in Ha, lengths in bohr.
* Cubic cell of edge ``a``; reciprocal lattice vectors b_i = (2 pi / a) e_i.
* Gamma-centred k grid, k = (i/N1, j/N2, l/N3) in reduced coordinates, i.e.
  every k has components in [0, 1).
* The state (n, k) is psi_nk(r) = Omega^-1/2 sum_{G in S_k} c_nk(G)
  e^{i(k+G).r} with S_k = {G : |k+G| < k_c} (k-centred sphere) and
  sum_G |c|^2 = 1; states are orthonormal within each k.
* Time reversal: let k' be the grid point of -k and G1 = k + k' (an integer
  vector).  Then c_{n k'}(G) = conj(c_{n k}(-G - G1)), eps_{n k'} = eps_{n k}
  and f_{n k'} = f_{n k}.  For a k that is its own partner (2k integer) the
  coefficients obey c(G) = conj(c(-G - 2k)); they are orthonormalised in the
  real coordinates in which that constraint is linear, which keeps it exact.

Random numbers come from numpy's PCG64 keyed by (seed, k index), so a k point's
draws do not depend on the order in which k points are built.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

HA_EV = 27.211386245988  # 1 Ha in eV (CODATA 2018)


@dataclasses.dataclass
class SystemSpec:
    a: float = 10.0                      # cubic cell edge (bohr)
    kgrid: tuple = (4, 4, 4)             # Gamma-centred Monkhorst-Pack grid
    n_occ: int = 8                       # occupied bands (insulating case)
    n_bands: int = 32                    # total bands per k
    kc: float = 2.6049                   # sphere radius |k+G| < kc (bohr^-1)
    fft: tuple = (24, 24, 24)            # real-space grid used for rho
    ng: int = 59                         # number of response G vectors
    q_frac: tuple = ((0.25, 0.0, 0.0),)  # q points in reduced coordinates
    freqs: tuple = (0j,)                 # complex frequencies (Ha)
    eta: float = 0.1 / HA_EV             # broadening (Ha), +i eta retarded
    occ_ev: tuple = (-10.0, 0.0)         # occupied energies, uniform (eV)
    emp_ev: tuple = (1.1, 30.0)          # empty energies, uniform (eV)
    kT_ev: Optional[float] = None        # None: 0/1 occupations; else Fermi-Dirac
    n_electrons: Optional[int] = None    # electrons per cell (Fermi-Dirac case)
    seed: int = 1
    coef_dtype: str = "c128"             # "c128" or "c64"
    spin_factor: float = 2.0
    flat_bands: bool = False             # True: every k gets the band energies of k = 0


@dataclasses.dataclass
class System:
    spec: SystemSpec
    lattice: np.ndarray      # (3,3) rows a1, a2, a3 (bohr)
    omega_cell: float        # cell volume (bohr^3)
    kfrac: np.ndarray        # (nk, 3) reduced k
    npw: np.ndarray          # (nk,) int32
    gvec: np.ndarray         # (nk, npw_max, 3) int32, zero padded
    coef: np.ndarray         # (nk, nb, npw_max) complex, zero padded
    eps: np.ndarray          # (nk, nb) Ha
    occ: np.ndarray          # (nk, nb) in [0, 1] per spin channel
    q_frac: np.ndarray       # (nq, 3)
    freqs: np.ndarray        # (nw,) complex Ha
    eta: float
    spin_factor: float
    fft: tuple
    ng: int

    @property
    def nk(self) -> int:
        return self.kfrac.shape[0]

    @property
    def nb(self) -> int:
        return self.coef.shape[1]

    @property
    def npw_max(self) -> int:
        return self.coef.shape[2]

    def sphere(self, ik: int) -> np.ndarray:
        return self.gvec[ik, : self.npw[ik]]

    def coefs(self, ik: int) -> np.ndarray:
        return self.coef[ik, :, : self.npw[ik]]


def kgrid_fractions(kgrid: Sequence[int]) -> np.ndarray:
    n1, n2, n3 = kgrid
    out = np.empty((n1 * n2 * n3, 3))
    idx = 0
    for i in range(n1):
        for j in range(n2):
            for l in range(n3):
                out[idx] = (i / n1, j / n2, l / n3)
                idx += 1
    return out


def _kindex(i: int, j: int, l: int, kgrid) -> int:
    return (i * kgrid[1] + j) * kgrid[2] + l


def sphere_miller(kfrac: np.ndarray, a: float, kc: float) -> np.ndarray:
    """Integer G with |(2 pi / a)(k + G)| < kc, in lexicographic order."""
    r = kc * a / (2.0 * math.pi)
    m = int(math.ceil(r)) + 1
    rng = np.arange(-m, m + 1)
    gx, gy, gz = np.meshgrid(rng, rng, rng, indexing="ij")
    g = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    kg = g + kfrac[None, :]
    keep = (kg * kg).sum(axis=1) < r * r
    g = g[keep]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0]))
    return g[order].astype(np.int32)


def gauss_legendre_freqs(n: int, lo_ev: float, hi_ev: float) -> np.ndarray:
    """n imaginary frequencies i*w on the Gauss-Legendre nodes of [lo, hi] eV."""
    x, _ = np.polynomial.legendre.leggauss(n)
    w_ev = 0.5 * (hi_ev - lo_ev) * x + 0.5 * (hi_ev + lo_ev)
    return 1j * (w_ev / HA_EV)


def tr_partner(ik: int, kgrid) -> int:
    """Index of the grid point of -k."""
    return _tr_partner(ik, kgrid)


def _tr_partner(ik: int, kgrid) -> int:
    n1, n2, n3 = kgrid
    i, rem = divmod(ik, n2 * n3)
    j, l = divmod(rem, n3)
    return _kindex((-i) % n1, (-j) % n2, (-l) % n3, kgrid)


def _orthonormal_generic(rng: np.random.Generator, npw: int, nb: int) -> np.ndarray:
    z = rng.standard_normal((npw, nb)) + 1j * rng.standard_normal((npw, nb))
    q, _ = np.linalg.qr(z)
    return q.T.copy()  # (nb, npw), orthonormal rows


def _orthonormal_self_partner(rng, g: np.ndarray, two_k: np.ndarray, nb: int) -> np.ndarray:
    """Rows orthonormal and obeying c(G) = conj(c(-G - 2k)) exactly."""
    npw = g.shape[0]
    lookup = {tuple(v): i for i, v in enumerate(g.tolist())}
    partner = np.array([lookup[tuple((-v - two_k).tolist())] for v in g], dtype=np.int64)
    idx = np.arange(npw)
    fixed = np.nonzero(partner == idx)[0]
    reps = np.nonzero(partner > idx)[0]
    nreal = fixed.size + 2 * reps.size
    assert nreal == npw
    x = rng.standard_normal((nreal, nb))
    qr_, _ = np.linalg.qr(x)   # real orthonormal columns
    coef = np.zeros((nb, npw), dtype=np.complex128)
    nf = fixed.size
    coef[:, fixed] = qr_[:nf].T
    xr = qr_[nf: nf + reps.size].T
    yr = qr_[nf + reps.size:].T
    s = 1.0 / math.sqrt(2.0)
    coef[:, reps] = s * (xr + 1j * yr)
    coef[:, partner[reps]] = s * (xr - 1j * yr)
    return coef


def make_system(spec: SystemSpec) -> System:
    kgrid = tuple(int(v) for v in spec.kgrid)
    nk = kgrid[0] * kgrid[1] * kgrid[2]
    nb = spec.n_bands
    kfrac = kgrid_fractions(kgrid)
    spheres = [sphere_miller(kfrac[ik], spec.a, spec.kc) for ik in range(nk)]
    npw = np.array([s.shape[0] for s in spheres], dtype=np.int32)
    npw_max = int(npw.max())
    gvec = np.zeros((nk, npw_max, 3), dtype=np.int32)
    for ik, s in enumerate(spheres):
        gvec[ik, : s.shape[0]] = s
    cdt = np.complex64 if spec.coef_dtype == "c64" else np.complex128
    coef = np.zeros((nk, nb, npw_max), dtype=cdt)
    eps = np.zeros((nk, nb))
    done = np.zeros(nk, dtype=bool)
    for ik in range(nk):
        if done[ik]:
            continue
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, ik])))
        jk = _tr_partner(ik, kgrid)
        e_occ = np.sort(rng.uniform(spec.occ_ev[0], spec.occ_ev[1], spec.n_occ))
        e_emp = np.sort(rng.uniform(spec.emp_ev[0], spec.emp_ev[1], nb - spec.n_occ))
        e = np.concatenate([e_occ, e_emp]) / HA_EV
        g = spheres[ik]
        if jk == ik:
            two_k = np.rint(2.0 * kfrac[ik]).astype(np.int64)
            c = _orthonormal_self_partner(rng, g.astype(np.int64), two_k, nb)
            coef[ik, :, : g.shape[0]] = c
            eps[ik] = e
            done[ik] = True
            continue
        c = _orthonormal_generic(rng, g.shape[0], nb)
        coef[ik, :, : g.shape[0]] = c
        eps[ik] = e
        # partner: c_{k'}(G') = conj(c_k(-G' - G1)), G1 = k + k'
        g1 = np.rint(kfrac[ik] + kfrac[jk]).astype(np.int64)
        gp = spheres[jk].astype(np.int64)
        lookup = {tuple(v): i for i, v in enumerate(g.tolist())}
        src = np.array([lookup[tuple((-v - g1).tolist())] for v in gp], dtype=np.int64)
        coef[jk, :, : gp.shape[0]] = np.conj(c[:, src])
        eps[jk] = e
        done[ik] = done[jk] = True
    if spec.flat_bands:
        # dispersionless bands: the pole energies eps_m - eps_n repeat at every
        # k, the degenerate case of Appendix B's pole grouping
        eps[:] = eps[0][None, :]
    occ = _occupations(spec, eps)
    lattice = spec.a * np.eye(3)
    return System(
        spec=spec,
        lattice=lattice,
        omega_cell=float(spec.a ** 3),
        kfrac=kfrac,
        npw=npw,
        gvec=gvec,
        coef=coef,
        eps=eps,
        occ=occ,
        q_frac=np.array(spec.q_frac, dtype=np.float64).reshape(-1, 3),
        freqs=np.array(spec.freqs, dtype=np.complex128).reshape(-1),
        eta=float(spec.eta),
        spin_factor=float(spec.spin_factor),
        fft=tuple(int(v) for v in spec.fft),
        ng=int(spec.ng),
    )


def _occupations(spec: SystemSpec, eps: np.ndarray) -> np.ndarray:
    nk, nb = eps.shape
    if spec.kT_ev is None:
        occ = np.zeros((nk, nb))
        occ[:, : spec.n_occ] = 1.0
        return occ
    kT = spec.kT_ev / HA_EV
    n_el = spec.n_electrons if spec.n_electrons is not None else 2 * spec.n_occ
    target = n_el / spec.spin_factor  # states per k filled, averaged over k

    def fill(mu):
        x = np.clip((eps - mu) / kT, -700.0, 700.0)
        return (1.0 / (np.exp(x) + 1.0)).sum() / nk

    lo, hi = eps.min() - 50 * kT, eps.max() + 50 * kT
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if fill(mid) < target:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    x = np.clip((eps - mu) / kT, -700.0, 700.0)
    return 1.0 / (np.exp(x) + 1.0)


# --------------------------------------------------------------------------
# Named workloads (the sizes the method is exercised at)
# --------------------------------------------------------------------------

def cfg_plain_fp64(seed: int = 1) -> SystemSpec:
    """Plain FP64 case: 4x4x4 k, 8+24 bands, ~300 PW, FFT 24^3, N_G = 59,
    q = (1/4,0,0), static w = 0 with eta = 0.1 eV, complex128 coefficients."""
    return SystemSpec(a=10.0, kgrid=(4, 4, 4), n_occ=8, n_bands=32, kc=2.6049,
                      fft=(24, 24, 24), ng=59, q_frac=((0.25, 0.0, 0.0),),
                      freqs=(0j,), eta=0.1 / HA_EV, seed=seed, coef_dtype="c128")


def cfg_precision(seed: int = 2, nw: int = 32) -> SystemSpec:
    """Mixed-precision case: 8x8x8 k, 16+184 bands, ~2000 PW, FFT 48^3,
    N_G = 1000, q = (1/4,0,0), 32 imaginary frequencies on a Gauss-Legendre
    grid in [0, 100] eV, complex64 coefficients."""
    return SystemSpec(a=10.0, kgrid=(8, 8, 8), n_occ=16, n_bands=200, kc=4.9124,
                      fft=(48, 48, 48), ng=1000, q_frac=((0.25, 0.0, 0.0),),
                      freqs=tuple(gauss_legendre_freqs(nw, 0.0, 100.0)), eta=0.0,
                      seed=seed, coef_dtype="c64")


def cfg_large(seed: int = 6, kgrid=(12, 12, 12), nw: int = 64) -> SystemSpec:
    """Large case: 12x12x12 k, 24 occupied + 976 empty bands, ~4000 PW,
    FFT 72^3, N_G = 3000, 64 imaginary frequencies on a Gauss-Legendre grid
    in [0, 100] eV, the 8 q points (j/12, 0, 0), j = 1..8, complex64
    coefficients.  Its states are too many for the host-side generator of
    this module (1728 QR factorisations of 4000 x 1000): the benchmark
    generates them on the device by the same recipe; its energies come from
    large_energies."""
    q = tuple((j / float(kgrid[0]), 0.0, 0.0) for j in range(1, 9))
    return SystemSpec(a=10.0, kgrid=tuple(kgrid), n_occ=24, n_bands=1000, kc=6.1842,
                      fft=(72, 72, 72), ng=3000, q_frac=q,
                      freqs=tuple(gauss_legendre_freqs(nw, 0.0, 100.0)), eta=0.0,
                      seed=seed, coef_dtype="c64")


def large_energies(spec: SystemSpec) -> np.ndarray:
    """Band energies of every k (Ha) by the recipe of make_system: per TR pair
    one draw keyed by (seed, k), occupied ~ U[occ_ev] and empty ~ U[emp_ev],
    each sorted, shared by the pair."""
    kgrid = tuple(int(v) for v in spec.kgrid)
    nk = kgrid[0] * kgrid[1] * kgrid[2]
    nb = spec.n_bands
    eps = np.zeros((nk, nb))
    done = np.zeros(nk, dtype=bool)
    for ik in range(nk):
        if done[ik]:
            continue
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([spec.seed, ik])))
        e_occ = np.sort(rng.uniform(spec.occ_ev[0], spec.occ_ev[1], spec.n_occ))
        e_emp = np.sort(rng.uniform(spec.emp_ev[0], spec.emp_ev[1], nb - spec.n_occ))
        jk = _tr_partner(ik, kgrid)
        eps[ik] = eps[jk] = np.concatenate([e_occ, e_emp]) / HA_EV
        done[ik] = done[jk] = True
    return eps


def cfg_tiny(seed: int = 11, kgrid=(2, 2, 2), n_occ=3, n_bands=6, kc=None,
             fft=(12, 12, 12), ng=3, q_frac=((0.5, 0.0, 0.0),), freqs=(0j,),
             eta=0.1 / HA_EV, coef_dtype="c128", a=6.0, npw_target=20,
             kT_ev=None) -> SystemSpec:
    """Small systems for brute-force and invariant checks."""
    if kc is None:
        # radius (in units of 2 pi / a) holding about npw_target plane waves
        r = (3.0 * npw_target / (4.0 * math.pi)) ** (1.0 / 3.0)
        kc = r * 2.0 * math.pi / a
    return SystemSpec(a=a, kgrid=tuple(kgrid), n_occ=n_occ, n_bands=n_bands, kc=kc,
                      fft=tuple(fft), ng=ng, q_frac=tuple(tuple(q) for q in q_frac),
                      freqs=tuple(freqs), eta=eta, seed=seed, coef_dtype=coef_dtype,
                      kT_ev=kT_ev)


def make_plane_wave_system(spec: SystemSpec, e_fermi: float) -> System:
    """A free-electron crystal: band n at k is the n-th plane wave of S_k in
    order of |k+G| (ties by ascending G), with coefficient 1, energy
    |k+G|^2/2 (Ha) and occupation 1 below e_fermi, else 0."""
    kgrid = tuple(int(v) for v in spec.kgrid)
    nk = kgrid[0] * kgrid[1] * kgrid[2]
    nb = spec.n_bands
    kfrac = kgrid_fractions(kgrid)
    b = 2.0 * math.pi / spec.a
    spheres = [sphere_miller(kfrac[ik], spec.a, spec.kc) for ik in range(nk)]
    npw = np.array([s.shape[0] for s in spheres], dtype=np.int32)
    if npw.min() < nb:
        raise ValueError("sphere holds fewer plane waves than bands")
    npw_max = int(npw.max())
    gvec = np.zeros((nk, npw_max, 3), dtype=np.int32)
    coef = np.zeros((nk, nb, npw_max), dtype=np.complex128)
    eps = np.zeros((nk, nb))
    for ik, s in enumerate(spheres):
        gvec[ik, : s.shape[0]] = s
        kin = 0.5 * b * b * ((s + kfrac[ik][None, :]) ** 2).sum(axis=1)
        order = np.lexsort((s[:, 2], s[:, 1], s[:, 0], np.round(kin, 12)))[:nb]
        coef[ik, np.arange(nb), order] = 1.0
        eps[ik] = kin[order]
    occ = (eps < e_fermi).astype(np.float64)
    return System(spec=spec, lattice=spec.a * np.eye(3), omega_cell=float(spec.a ** 3),
                  kfrac=kfrac, npw=npw, gvec=gvec, coef=coef, eps=eps, occ=occ,
                  q_frac=np.array(spec.q_frac, dtype=np.float64).reshape(-1, 3),
                  freqs=np.array(spec.freqs, dtype=np.complex128).reshape(-1),
                  eta=float(spec.eta), spin_factor=float(spec.spin_factor),
                  fft=tuple(int(v) for v in spec.fft), ng=int(spec.ng))


def truncate_bands(system: System, nb: int) -> System:
    """The same crystal described with only its first nb bands (coefficients,
    energies and occupations of bands 0..nb-1)."""
    spec = dataclasses.replace(system.spec, n_bands=nb)
    return dataclasses.replace(system, spec=spec, coef=np.ascontiguousarray(system.coef[:, :nb]),
                               eps=np.ascontiguousarray(system.eps[:, :nb]),
                               occ=np.ascontiguousarray(system.occ[:, :nb]))


def _smooth_at_least(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n (FFT-friendly grid size)."""
    m = n
    while True:
        r = m
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        if r == 1:
            return m
        m += 1


def make_batching_system(s: int, nq_max=None, coef_dtype: str = "c64") -> System:
    """System s of the batching workload (seed 3000 + s): cell edge a ~ U[8, 14]
    bohr, 4x4x4 k, plane waves per state log-uniform on [400, 4000] (sphere
    radius from the count), N_G ~ U{200..1500}, N_q ~ U{4..20} distinct nonzero
    grid vectors, N_w ~ U{8..64} imaginary frequencies on the Gauss-Legendre
    nodes of [0, 100] eV, 64 bands with energies ~ U[-10, 30] eV sorted per k,
    Fermi-Dirac occupations at kT = 0.05 eV for 32 electrons per cell (metals:
    transition counts differ from k to k).  The FFT grid is the smallest
    2^a 3^b 5^c at least 4 n_max + 1 (n_max the largest Miller index of the
    spheres) and alias free for the response set.  nq_max keeps only the first
    nq_max q vectors."""
    rng = np.random.default_rng(3000 + s)
    a = float(rng.uniform(8.0, 14.0))
    npw = float(np.exp(rng.uniform(np.log(400.0), np.log(4000.0))))
    kc = (3.0 * npw / (4.0 * math.pi)) ** (1.0 / 3.0) * 2.0 * math.pi / a
    ng = int(rng.integers(200, 1501))
    nq = int(rng.integers(4, 21))
    nw = int(rng.integers(8, 65))
    grid = [(i, j, l) for i in range(4) for j in range(4) for l in range(4) if (i, j, l) != (0, 0, 0)]
    pick = rng.choice(len(grid), size=nq, replace=False)
    qs = tuple(tuple(v / 4.0 for v in grid[p]) for p in pick)
    if nq_max is not None:
        qs = qs[:nq_max]
    spec = SystemSpec(a=a, kgrid=(4, 4, 4), n_occ=0, n_bands=64, kc=kc, fft=(8, 8, 8), ng=ng, q_frac=qs,
                      freqs=tuple(gauss_legendre_freqs(nw, 0.0, 100.0)), eta=0.0, occ_ev=(-10.0, 30.0),
                      emp_ev=(-10.0, 30.0), kT_ev=0.05, n_electrons=32, seed=3000 + s, coef_dtype=coef_dtype)
    sysm = make_system(spec)
    n_max = int(np.abs(sysm.gvec).max())
    r_g = (3.0 * ng / (4.0 * math.pi)) ** (1.0 / 3.0) + 2.0      # response-set extent, with margin
    n = _smooth_at_least(max(4 * n_max + 1, 2 * n_max + int(math.ceil(r_g)) + 3))
    spec = dataclasses.replace(spec, fft=(n, n, n))
    return dataclasses.replace(sysm, spec=spec, fft=(n, n, n))


def cfg_learned(seed: int = 4000, full_bands: int = 800, n_occ: int = 12, kgrid=(6, 6, 6),
                kc: float = 4.4601, fft=(32, 32, 32), ng: int = 500, nw: int = 16) -> SystemSpec:
    """Learned-terminator case: 6x6x6 k, 12 occupied bands, ~1500 PW, FFT 32^3,
    N_G = 500, q = (1/6,0,0), 16 imaginary frequencies on [0, 100] eV; the
    truncated chi0 uses the first bands of the same system.  Smaller variants
    (for tests) override the keyword arguments."""
    q = (1.0 / kgrid[0], 0.0, 0.0)
    return SystemSpec(a=10.0, kgrid=tuple(kgrid), n_occ=n_occ, n_bands=full_bands, kc=kc,
                      fft=tuple(fft), ng=ng, q_frac=(q,), freqs=tuple(gauss_legendre_freqs(nw, 0.0, 100.0)),
                      eta=0.0, seed=seed, coef_dtype="c64")


def make_closure_system(seed: int = 5, L: int = 3, L_occ: int = 1, n_occ: int = 2, nb_keep: int = 12,
                        omitted_ev=(45.0, 45.0), ng: int = 7, fft=(16, 16, 16),
                        freqs=(0.3j, 2.0j), coef_dtype: str = "c128") -> System:
    """A two-k system whose band basis is complete: at each k the plane waves
    are every G with |G_a| <= L and there are as many bands, from a random
    unitary matrix.  The occupied bands are built from G with |G_a| <= L_occ
    only, so with response vectors and umklapp vectors within |G_a| <= 1 every
    product of an occupied state with e^{i(q+G).r} stays inside the basis.
    Energies: occupied uniform in [-10, 0] eV, bands n_occ..nb_keep-1 uniform
    in [1, 30] eV (sorted), the rest uniform in omitted_ev (eV; equal ends put
    them all at one energy).  q = (1/2, 0, 0) on a 2 x 1 x 1 grid.  No
    time-reversal pairing is imposed: the identities this system serves
    (closure over a complete band set) do not need it."""
    rng = np.random.default_rng(seed)
    v = np.arange(-L, L + 1)
    g = np.stack(np.meshgrid(v, v, v, indexing="ij"), axis=-1).reshape(-1, 3)
    npw = g.shape[0]
    inner = np.nonzero(np.all(np.abs(g) <= L_occ, axis=1))[0]
    nk = 2
    coef = np.zeros((nk, npw, npw), dtype=np.complex128)
    eps = np.zeros((nk, npw))
    occ = np.zeros((nk, npw))
    for ik in range(nk):
        M = rng.standard_normal((npw, npw)) + 1j * rng.standard_normal((npw, npw))
        M[:, :n_occ] = 0.0
        M[inner, :n_occ] = (rng.standard_normal((inner.size, n_occ))
                            + 1j * rng.standard_normal((inner.size, n_occ)))
        Q, _ = np.linalg.qr(M)  # orthonormal columns, the first n_occ on the inner cube
        coef[ik] = Q.T
        eps[ik, :n_occ] = rng.uniform(-10.0, 0.0, n_occ) / HA_EV
        eps[ik, n_occ:nb_keep] = np.sort(rng.uniform(1.0, 30.0, nb_keep - n_occ)) / HA_EV
        eps[ik, nb_keep:] = rng.uniform(omitted_ev[0], omitted_ev[1], npw - nb_keep) / HA_EV
        occ[ik, :n_occ] = 1.0
    if coef_dtype == "c64":
        coef = coef.astype(np.complex64)
    spec = SystemSpec(a=6.0, kgrid=(2, 1, 1), n_occ=n_occ, n_bands=npw, fft=tuple(fft), ng=ng,
                      q_frac=((0.5, 0.0, 0.0),), freqs=tuple(freqs), eta=0.0, seed=seed, coef_dtype=coef_dtype)
    return System(spec=spec, lattice=6.0 * np.eye(3), omega_cell=216.0,
                  kfrac=np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]]), npw=np.full(nk, npw, dtype=np.int32),
                  gvec=np.broadcast_to(g, (nk, npw, 3)).astype(np.int32).copy(), coef=coef, eps=eps, occ=occ,
                  q_frac=np.array(spec.q_frac), freqs=np.array(spec.freqs), eta=0.0, spin_factor=2.0,
                  fft=spec.fft, ng=spec.ng)
