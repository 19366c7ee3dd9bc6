"""Three-body amplitude (Dalitz-plot) model, float64 / complex128, CPU.

The paper lists dedicated amplitude-analysis PDFs for three-body decays among GooFit's
PDFs (Sec. 1), notes that some components are complex amplitudes whose squared magnitude is
the density (Sec. 1, footnote), and uses MC phase-space samples for the normalisation
integral (Sec. 5).  No formula is printed, so this file writes out the
standard isobar model:

  particles 1, 2, 3 of masses m1, m2, m3 from a parent of mass M; observables s12, s13;
  s23 = M^2 + m1^2 + m2^2 + m3^2 - s12 - s13.
  For a resonance R in pair (A, B) with bachelor C and s = s_AB:
    q(s)   = momentum of A in the R rest frame    = sqrt(lambda(s, mA^2, mB^2)) / (2 sqrt s)
    k(s)   = momentum of C in the R rest frame
    p*(s)  = momentum of C in the parent rest frame = sqrt(lambda(M^2, s, mC^2)) / (2 M)
    cos(theta) = cosine of the angle between A and C in the R rest frame
    Blatt-Weisskopf barrier, z = (r q)^2, normalised to 1 at z = 0:
        B0 = 1,  B1 = sqrt(1/(1+z)),  B2 = sqrt(9/(9 + 3z + z^2))
    running width  Gamma(s) = G0 (q/q0)^(2L+1) (m0/sqrt s) (B_L(z)/B_L(z0))^2,  q0 = q(m0^2)
    Breit-Wigner   BW(s) = 1 / (m0^2 - s - i m0 Gamma(s))
    spin factor    Z0 = 1,  Z1 = -4 q k cos(theta),  Z2 = 16 q^2 k^2 (cos^2(theta) - 1/3)
    amplitude      A_R = BW(s) * B_L(r_res q)/B_L(r_res q0) * B_L(r_par p*) * Z_L
  the non-resonant amplitude is A_NR = 1.
  Total amplitude S = sum_k c_k A_k with complex coefficients c_k = Re_k + i Im_k.
  Density f = |S|^2 / N,  N = mean over a uniform phase-space MC sample of |S|^2
  (the constant phase-space volume is dropped; it does not depend on theta).
  NLL = - sum_i log f(x_i).

The spin factor is computed here from the helicity angle; the CUDA path uses the
equivalent invariant-mass expression, and tests/test_oracle_dalitz.py pins the two
against each other and against explicit four-vector kinematics.
"""
import torch

PAIRS = {  # pair -> (A, B, C) particle indices
    "12": (1, 2, 3),
    "13": (1, 3, 2),
    "23": (2, 3, 1),
}


def kallen(a, b, c):
    return a * a + b * b + c * c - 2 * a * b - 2 * a * c - 2 * b * c


def invariants(s12, s13, M, m1, m2, m3):
    s23 = M * M + m1 * m1 + m2 * m2 + m3 * m3 - s12 - s13
    return {"12": s12, "13": s13, "23": s23}


def pair_masses(pair, masses):
    a, b, c = PAIRS[pair]
    return masses[a], masses[b], masses[c]


def s_of(inv, i, j):
    key = f"{min(i, j)}{max(i, j)}"
    return inv[key]


def barrier(L, z):
    if L == 0:
        return torch.ones_like(z)
    if L == 1:
        return torch.sqrt(1.0 / (1.0 + z))
    if L == 2:
        return torch.sqrt(9.0 / (9.0 + 3.0 * z + z * z))
    raise ValueError("spin > 2 not supported")


def helicity_frame(s, s_ac, M, mA, mB, mC):
    """(q, k, cos theta) in the rest frame of the (A B) pair of mass sqrt(s)."""
    rs = torch.sqrt(s)
    eA = (s + mA * mA - mB * mB) / (2 * rs)
    eC = (M * M - s - mC * mC) / (2 * rs)
    q = torch.sqrt(torch.clamp(kallen(s, mA * mA, mB * mB), min=0.0)) / (2 * rs)
    k = torch.sqrt(torch.clamp(eC * eC - mC * mC, min=0.0))
    cos = (mA * mA + mC * mC + 2 * eA * eC - s_ac) / (2 * q * k)
    return q, k, cos


def spin_factor(L, q, k, cos):
    if L == 0:
        return torch.ones_like(q)
    if L == 1:
        return -4.0 * q * k * cos
    if L == 2:
        return 16.0 * q * q * k * k * (cos * cos - 1.0 / 3.0)
    raise ValueError("spin > 2 not supported")


def resonance_amplitude(s12, s13, kin, pair, L, m0, g0, dtype=torch.float64):
    M = kin["M"]
    masses = {1: kin["m1"], 2: kin["m2"], 3: kin["m3"]}
    inv = invariants(s12, s13, M, kin["m1"], kin["m2"], kin["m3"])
    a, b, c = PAIRS[pair]
    mA, mB, mC = masses[a], masses[b], masses[c]
    s = s_of(inv, a, b)
    s_ac = s_of(inv, a, c)
    q, k, cos = helicity_frame(s, s_ac, M, mA, mB, mC)
    m0 = torch.as_tensor(m0, dtype=dtype)
    g0 = torch.as_tensor(g0, dtype=dtype)
    q0 = torch.sqrt(kallen(m0 * m0, mA * mA, mB * mB)) / (2 * m0)
    r = kin["r_res"]
    ratio = barrier(L, (r * q) ** 2) / barrier(L, (r * q0) ** 2)
    bw = breit_wigner(s, m0, g0, L, q, q0, r)
    pstar = torch.sqrt(torch.clamp(kallen(M * M, s, mC * mC), min=0.0)) / (2 * M)
    parent = barrier(L, (kin["r_par"] * pstar) ** 2)
    return bw * (ratio * parent * spin_factor(L, q, k, cos))


def running_width(s, m0, g0, L, q, q0, r):
    ratio = barrier(L, (r * q) ** 2) / barrier(L, (r * q0) ** 2)
    return g0 * (q / q0) ** (2 * L + 1) * (m0 / torch.sqrt(s)) * ratio ** 2


def breit_wigner(s, m0, g0, L, q, q0, r):
    """Relativistic Breit--Wigner 1 / (m0^2 - s - i m0 Gamma(s)) with the running width."""
    return 1.0 / torch.complex(m0 * m0 - s, -m0 * running_width(s, m0, g0, L, q, q0, r))


def inside(s12, s13, kin):
    """Physical-region test: |cos theta| <= 1 for the (12) pair with s12 above threshold."""
    s12 = torch.as_tensor(s12, dtype=torch.float64)
    s13 = torch.as_tensor(s13, dtype=torch.float64)
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    ok = (s12 > (m1 + m2) ** 2) & (s12 < (M - m3) ** 2)
    s12c = torch.clamp(s12, (m1 + m2) ** 2 + 1e-12, (M - m3) ** 2 - 1e-12)
    _, _, cos = helicity_frame(s12c, s13, M, m1, m2, m3)
    return ok & (cos.abs() <= 1.0)


class DalitzModel:
    """The spec's ("coherent", kin, amps) tree."""

    def __init__(self, spec):
        assert spec["pdf"][0] == "coherent"
        self.spec = spec
        self.kin = spec["pdf"][1]
        self.amps = spec["pdf"][2]
        self.pidx = {p[0]: i for i, p in enumerate(spec["params"])}

    def amplitude_matrix(self, cols, theta, dtype=torch.float64):
        """Complex [n_events, K] matrix of the amplitudes A_k (coefficients not applied)."""
        th = torch.as_tensor(theta, dtype=dtype) if not torch.is_tensor(theta) else theta.to(dtype)
        s12 = torch.as_tensor(cols["s12"], dtype=dtype)
        s13 = torch.as_tensor(cols["s13"], dtype=dtype)
        out = []
        for amp in self.amps:
            if amp[0] == "bw":
                _, pair, L, m0n, g0n, _, _ = amp
                out.append(resonance_amplitude(s12, s13, self.kin, pair, L,
                                               th[self.pidx[m0n]], th[self.pidx[g0n]], dtype=dtype))
            elif amp[0] == "nr":
                out.append(torch.complex(torch.ones_like(s12), torch.zeros_like(s12)))
            else:
                raise ValueError(amp[0])
        return torch.stack(out, dim=1)

    def coefficients(self, th):
        """c_k from the two parameters of amplitude k: (Re, Im), or with spec["coef"] ==
        "polar" (magnitude r, phase phi): c = r (cos phi + i sin phi)."""
        u = torch.stack([th[self.pidx[a[-2]]] for a in self.amps])
        v = torch.stack([th[self.pidx[a[-1]]] for a in self.amps])
        if self.spec.get("coef") == "polar":
            return torch.complex(u * torch.cos(v), u * torch.sin(v))
        return torch.complex(u, v)

    def intensity(self, A, th):
        S = A @ self.coefficients(th)
        return S.real ** 2 + S.imag ** 2

    def nll_grad(self, cols, mc_cols, theta):
        th = torch.tensor([float(t) for t in theta], dtype=torch.float64, requires_grad=True)
        A = self.amplitude_matrix(cols, th)
        Amc = self.amplitude_matrix(mc_cols, th)
        norm = self.intensity(Amc, th).mean()
        nll = -torch.log(self.intensity(A, th) / norm).sum()
        (g,) = torch.autograd.grad(nll, th)
        return float(nll.detach()), g.numpy().copy()

    def nll(self, cols, mc_cols, theta):
        with torch.no_grad():
            th = torch.as_tensor(theta, dtype=torch.float64)
            norm = self.intensity(self.amplitude_matrix(mc_cols, th), th).mean()
            return float(-torch.log(self.intensity(self.amplitude_matrix(cols, th), th) / norm).sum())

    def density(self, cols, mc_cols, theta):
        with torch.no_grad():
            th = torch.as_tensor(theta, dtype=torch.float64)
            norm = self.intensity(self.amplitude_matrix(mc_cols, th), th).mean()
            return self.intensity(self.amplitude_matrix(cols, th), th) / norm

    def gram(self, mc_cols, theta):
        """G_kl = mean over the MC sample of A_k conj(A_l)."""
        with torch.no_grad():
            A = self.amplitude_matrix(mc_cols, theta)
            return (A.T @ A.conj()) / A.shape[0]


def max_intensity_scan(model, theta, n=400):
    """Largest |S|^2 over an n x n grid of the physical region (for accept--reject envelopes)."""
    kin = model.kin
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    a = torch.linspace((m1 + m2) ** 2, (M - m3) ** 2, n, dtype=torch.float64)
    b = torch.linspace((m1 + m3) ** 2, (M - m2) ** 2, n, dtype=torch.float64)
    A, B = torch.meshgrid(a, b, indexing="ij")
    A, B = A.reshape(-1), B.reshape(-1)
    ok = inside(A, B, kin)
    cols = {"s12": A[ok], "s13": B[ok]}
    with torch.no_grad():
        th = torch.as_tensor(theta, dtype=torch.float64)
        return float(model.intensity(model.amplitude_matrix(cols, th), th).max())

