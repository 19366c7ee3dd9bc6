"""Model specifications (plain data) for the five synthetic workloads.

A spec is a dict:
  name         workload name
  observables  [(name, lo, hi), ...]           event columns, in column order
  params       [(name, value, fixed, step), ...] parameter vector theta, in order
  pdf          expression tree (tuples, see below)
  norm         ("analytic",) | ("grid", [bins per observable]) | ("mc", n_points, seed)

Tree nodes (parameter and observable references are names):
  ("gauss", obs, mu, sigma)        ("expo", obs, lam)
  ("poly2", obs, a1, a2)           ("argus", obs, m0, c, p)
  ("prod", [child, ...])           ("add", [frac, ...], [child, ...])   K children, K-1 fractions
  ("coherent", kin, [amp, ...])    kin = dict(M, m1, m2, m3, r_res, r_par)
      amp = ("bw", pair, spin, m0, width, re, im) | ("nr", re, im);  pair in {"12","13","23"}
  ("td4", kin, [amp, ...], (x, y, tau, sigma_t))   kin = dict(M, m1, m2, m3, m4, r_res)
      amp = (angular, (m0, width) in pair 12, (m0, width) in pair 34, re, im, (cf_re, cf_im))
      observables in the order m12, m34, cos th12, cos th34, phi, t

The paper (GooFit 2.0, Fig. 1 and Sec. 1) describes models built from basic PDFs combined
by sum and product combination PDFs and amplitude PDFs for three-body decays (Sec. 1,
Sec. 5); it prints no formulas, so the meaning of each node is fixed by the oracle.
"""
import math

# Parent and daughter masses (GeV) of the D -> K pi pi0 - like three-body model.
DALITZ_MASSES = dict(M=1.865, m1=0.494, m2=0.140, m3=0.135)


def c1_spec():
    """1D: 0.3 Gauss(5.0, 0.4) + 0.7 Exp(-0.3) on x in [0, 10], analytic normalisation."""
    return dict(
        name="c1_1d",
        observables=[("x", 0.0, 10.0)],
        params=[("mu", 5.0, False, 0.01), ("sigma", 0.4, False, 0.01),
                ("lam", -0.3, False, 0.005), ("frac", 0.3, False, 0.005)],
        pdf=("add", ["frac"], [("gauss", "x", "mu", "sigma"), ("expo", "x", "lam")]),
        norm=("analytic",),
    )


def c2_spec(bins=128):
    """3D: 0.2 [Gauss(m) Gauss(dE) Exp(t)] + 0.8 [Argus(m) Poly2(dE) Exp(t)], grid normalisation."""
    return dict(
        name="c2_3d",
        observables=[("m", 5.2, 5.3), ("dE", -0.2, 0.2), ("t", 0.0, 10.0)],
        params=[("mu_m", 5.279, False, 1e-4), ("sig_m", 0.003, False, 1e-4),
                ("mu_de", 0.0, False, 1e-3), ("sig_de", 0.02, False, 1e-3),
                ("lam_s", -1.0 / 1.5, False, 1e-2),
                ("m0", 5.29, False, 1e-4), ("c", -20.0, False, 0.5), ("p", 0.5, False, 0.02),
                ("a1", -1.0, False, 0.05), ("a2", 0.5, False, 0.2),
                ("lam_b", -1.0 / 0.8, False, 1e-2), ("frac", 0.2, False, 1e-3)],
        pdf=("add", ["frac"], [
            ("prod", [("gauss", "m", "mu_m", "sig_m"), ("gauss", "dE", "mu_de", "sig_de"),
                      ("expo", "t", "lam_s")]),
            ("prod", [("argus", "m", "m0", "c", "p"), ("poly2", "dE", "a1", "a2"),
                      ("expo", "t", "lam_b")]),
        ]),
        norm=("grid", [bins, bins, bins]),
    )


def dalitz_resonances():
    """The eight resonances of the three-body model: (name, pair, spin, m0, width).

    Particle labels: 1 = K, 2 = pi, 3 = pi0.  Masses and widths are PDG-like round values.
    """
    return [
        ("Kst892_12", "12", 1, 0.8955, 0.0473),
        ("Kst892_13", "13", 1, 0.8955, 0.0473),
        ("rho770_23", "23", 1, 0.7753, 0.1491),
        ("K0st1430_12", "12", 0, 1.425, 0.270),
        ("K0st1430_13", "13", 0, 1.425, 0.270),
        ("K2st1430_12", "12", 2, 1.4324, 0.109),
        ("Kst1680_12", "12", 1, 1.718, 0.322),
        ("rho1450_23", "23", 1, 1.465, 0.400),
    ]


# Truth coefficients (Re, Im) of the eight resonant amplitudes; the non-resonant
# amplitude is the fixed reference c = (1, 0).
DALITZ_TRUTH = [
    (0.913, 0.303), (-0.456, 0.580), (0.999, -0.447), (0.585, 0.400),
    (-0.411, 0.366), (1.252, -0.293), (1.726, 1.725), (-0.918, 1.725),
]


def c3_spec(n_mc=1_000_000, mc_seed=1710013):
    """Three-body Dalitz model: 8 Breit--Wigner resonances + constant NR, 16 free coefficients."""
    kin = dict(DALITZ_MASSES, r_res=1.5, r_par=5.0)
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    params, amps = [], []
    for (name, pair, spin, m0, w), (re, im) in zip(dalitz_resonances(), DALITZ_TRUTH):
        params += [(f"m0_{name}", m0, True, 0.0), (f"w_{name}", w, True, 0.0),
                   (f"re_{name}", re, False, 0.02), (f"im_{name}", im, False, 0.02)]
        amps.append(("bw", pair, spin, f"m0_{name}", f"w_{name}", f"re_{name}", f"im_{name}"))
    params += [("re_NR", 1.0, True, 0.0), ("im_NR", 0.0, True, 0.0)]
    amps.append(("nr", "re_NR", "im_NR"))
    return dict(
        name="c3_dalitz",
        observables=[("s12", (m1 + m2) ** 2, (M - m3) ** 2), ("s13", (m1 + m3) ** 2, (M - m2) ** 2)],
        params=params,
        pdf=("coherent", kin, amps),
        norm=("mc", n_mc, mc_seed),
    )


# Parent and daughter masses (GeV) of the D -> K pi pi pi - like four-body model; particles
# 1 = K, 2 = pi (the K pi pair "12"), 3, 4 = pi pi (the pair "34").
TD4_MASSES = dict(M=1.865, m1=0.494, m2=0.140, m3=0.140, m4=0.140)

# Two-body resonances (m0, width in GeV) of the four-body model.
TD4_RESONANCES = {
    "Kst892": (0.8955, 0.0473), "K0st1430": (1.425, 0.270), "K2st1430": (1.4324, 0.109),
    "Kst1410": (1.414, 0.232), "rho770": (0.7753, 0.1491), "f0980": (0.990, 0.070),
    "rho1450": (1.465, 0.400),
}

# The ten amplitudes: (name, angular structure, resonance in pair 12, resonance in pair 34,
# truth of the free DCS coefficient (Re, Im), fixed CF coefficient (Re, Im)).  Angular
# structures (spins of the two resonances in brackets):
#   SS  (0,0): 1                     VS0 (1,0): cos th12          SV0 (0,1): cos th34
#   VV0 (1,1): cos th12 cos th34     VVpar (1,1): sin th12 sin th34 cos phi
#   VVperp (1,1): i sin th12 sin th34 sin phi
#   TS0 (2,0): (3 cos^2 th12 - 1)/2  TV0 (2,1): (3 cos^2 th12 - 1)/2 cos th34
TD4_AMPS = [
    ("KstRho_0", "VV0", "Kst892", "rho770", (1.0, 0.0), (0.9, 0.3)),
    ("KstRho_par", "VVpar", "Kst892", "rho770", (0.45, 0.2), (0.3, -0.1)),
    ("KstRho_perp", "VVperp", "Kst892", "rho770", (-0.3, 0.25), (0.2, 0.3)),
    ("KstF0", "VS0", "Kst892", "f0980", (0.35, -0.15), (-0.4, 0.2)),
    ("K0stRho", "SV0", "K0st1430", "rho770", (0.5, 0.3), (0.45, 0.1)),
    ("K0stF0", "SS", "K0st1430", "f0980", (0.25, -0.4), (0.3, 0.25)),
    ("K2stRho", "TV0", "K2st1430", "rho770", (0.3, 0.1), (-0.25, 0.2)),
    ("K2stF0", "TS0", "K2st1430", "f0980", (-0.2, 0.15), (0.2, -0.1)),
    ("Kst1410Rho", "VV0", "Kst1410", "rho770", (0.4, -0.25), (0.35, 0.2)),
    ("KstRho1450", "VV0", "Kst892", "rho1450", (0.3, 0.35), (0.25, -0.3)),
]

# Mixing and time-resolution truth: x, y, lifetime tau (ps), Gaussian resolution sigma_t (ps).
TD4_TIME = dict(x=0.004, y=0.006, tau=0.41, sigma_t=0.05)


def c4_spec(n_mc=3_000_000, mc_seed=1710014):
    """Time-dependent four-body model: 10 amplitudes, 20 free DCS coefficients, x, y, tau, sigma_t."""
    kin = dict(TD4_MASSES, r_res=1.5)
    M, m1, m2, m3, m4 = kin["M"], kin["m1"], kin["m2"], kin["m3"], kin["m4"]
    params, amps = [], []
    for name, ang, r12, r34, (re, im), (cre, cim) in TD4_AMPS:
        params += [(f"re_{name}", re, False, 0.02), (f"im_{name}", im, False, 0.02)]
        amps.append((ang, TD4_RESONANCES[r12], TD4_RESONANCES[r34], f"re_{name}", f"im_{name}", (cre, cim)))
    params += [("x", TD4_TIME["x"], False, 0.002), ("y", TD4_TIME["y"], False, 0.002),
               ("tau", TD4_TIME["tau"], False, 0.002), ("sigma_t", TD4_TIME["sigma_t"], False, 0.001)]
    return dict(
        name="c4_td4",
        observables=[("m12", m1 + m2, M - m3 - m4), ("m34", m3 + m4, M - m1 - m2), ("c12", -1.0, 1.0),
                     ("c34", -1.0, 1.0), ("phi", -math.pi, math.pi), ("t", -0.5, 10.0)],
        params=params,
        pdf=("td4", kin, amps, ("x", "y", "tau", "sigma_t")),
        norm=("mc", n_mc, mc_seed),
    )


# Time-dependent three-body model (D0 -> pi+ pi- pi0-like): particle 1 = pi0, 2 = pi+,
# 3 = pi- (equal charged-pion masses, so the Dalitz plot is symmetric under s12 <-> s13).
TD3_MASSES = dict(M=1.865, m1=0.1350, m2=0.1396, m3=0.1396)

# The fifteen Breit--Wigner amplitudes (name, pair, spin, m0, width): rho-like vectors in all
# three pairs and scalar/tensor states in the charged pair "23", with PDG-like round values.
TD3_RESONANCES = [
    ("rho770_p", "12", 1, 0.7753, 0.1491), ("rho770_m", "13", 1, 0.7753, 0.1491),
    ("rho770_0", "23", 1, 0.7753, 0.1491), ("rho1450_p", "12", 1, 1.465, 0.400),
    ("rho1450_m", "13", 1, 1.465, 0.400), ("rho1450_0", "23", 1, 1.465, 0.400),
    ("rho1700_p", "12", 1, 1.720, 0.250), ("rho1700_m", "13", 1, 1.720, 0.250),
    ("rho1700_0", "23", 1, 1.720, 0.250), ("f0_980", "23", 0, 0.990, 0.070),
    ("f2_1270", "23", 2, 1.2755, 0.1867), ("f0_1370", "23", 0, 1.350, 0.350),
    ("f0_1500", "23", 0, 1.505, 0.109), ("f0_500", "23", 0, 0.500, 0.400),
    ("f0_1710", "23", 0, 1.720, 0.135),
]

# Coefficient truth values (Re, Im): the rho+(770) is the fixed reference (1, 0); the last
# entry is the non-resonant amplitude.
TD3_TRUTH = [
    (1.0, 0.0), (0.55, 0.45), (0.52, 0.28), (0.35, -0.25), (0.30, 0.35), (0.20, 0.10),
    (0.25, 0.30), (-0.20, 0.30), (0.15, -0.20), (0.12, 0.05), (0.25, 0.15), (0.20, -0.10),
    (0.10, 0.08), (0.30, 0.20), (0.06, -0.04), (0.50, 0.20),
]


def td3_spec(n_mc=1_000_000, mc_seed=1710015):
    """Time-dependent three-body model: 15 BW + NR amplitudes (30 free coefficients, the
    rho+(770) the reference), x, y, tau, sigma_t; observables s12, s13, t."""
    kin = dict(TD3_MASSES, r_res=1.5, r_par=5.0)
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    params, amps = [], []
    for k, ((name, pair, spin, m0, w), (re, im)) in enumerate(zip(TD3_RESONANCES, TD3_TRUTH)):
        fixed = k == 0
        params += [(f"m0_{name}", m0, True, 0.0), (f"w_{name}", w, True, 0.0),
                   (f"re_{name}", re, fixed, 0.0 if fixed else 0.02),
                   (f"im_{name}", im, fixed, 0.0 if fixed else 0.02)]
        amps.append(("bw", pair, spin, f"m0_{name}", f"w_{name}", f"re_{name}", f"im_{name}"))
    re, im = TD3_TRUTH[-1]
    params += [("re_NR", re, False, 0.02), ("im_NR", im, False, 0.02)]
    amps.append(("nr", "re_NR", "im_NR"))
    params += [("x", TD4_TIME["x"], False, 0.002), ("y", TD4_TIME["y"], False, 0.002),
               ("tau", TD4_TIME["tau"], False, 0.002), ("sigma_t", TD4_TIME["sigma_t"], False, 0.001)]
    return dict(
        name="td3_dalitz",
        observables=[("s12", (m1 + m2) ** 2, (M - m3) ** 2), ("s13", (m1 + m3) ** 2, (M - m2) ** 2),
                     ("t", -0.5, 10.0)],
        params=params,
        pdf=("td3", kin, amps, ("x", "y", "tau", "sigma_t")),
        norm=("mc", n_mc, mc_seed),
    )


def to_polar(spec):
    """The same amplitude model with each complex coefficient parameterised by its magnitude
    and phase: parameters re_X / im_X become mag_X / phase_X (values |c|, arg c; steps scaled
    alike), spec["coef"] = "polar"."""
    vals = {p[0]: p for p in spec["params"]}
    ren, params = {}, []
    for p in spec["params"]:
        if p[0].startswith("re_") and "im_" + p[0][3:] in vals:
            q = vals["im_" + p[0][3:]]
            c = complex(p[1], q[1])
            r, ph = abs(c), math.atan2(c.imag, c.real)
            ren[p[0]], ren[q[0]] = "mag_" + p[0][3:], "phase_" + p[0][3:]
            params.append((ren[p[0]], r, p[2], p[3]))
            params.append((ren[q[0]], ph, q[2], p[3] / max(r, 1e-3) if p[3] > 0 else 0.0))
        elif not p[0].startswith("im_"):
            params.append(p)
    kind = spec["pdf"][0]
    amps = [tuple(ren.get(x, x) if isinstance(x, str) else x for x in a) for a in spec["pdf"][2]]
    pdf = (kind, spec["pdf"][1], amps) + tuple(spec["pdf"][3:])
    return dict(spec, params=params, pdf=pdf, coef="polar")


def param_names(spec):
    return [p[0] for p in spec["params"]]


def param_values(spec):
    return [float(p[1]) for p in spec["params"]]


def observable_names(spec):
    return [o[0] for o in spec["observables"]]
