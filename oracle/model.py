"""Composite-PDF semantics, normalisation and the unbinned NLL (float64, CPU).

Reading of the paper (Fig. 1 caption; Sec. 1: basic PDFs put together by combination
PDFs and fitted by a FitManager to an unbinned DataSet, following RooFit, Sec. 1):

  shape(leaf)  = the leaf's unnormalised shape u(x)                 (oracle/pdfs.py)
  shape(PROD)  = product of the children's shapes; the children act on disjoint observables
  shape(ADD)   = sum_k w_k shape(child_k) / norm(child_k),  w_k = frac_k for k < K-1,
                 w_{K-1} = 1 - sum of the K-1 fractions            (fractions of normalised
                 components: an ADD is itself normalised)
  norm(ADD)    = 1
  norm(node)   analytic mode: leaf -> closed-form integral over its range,
                              PROD -> product of the children's norms
               grid mode:     integral of shape(node) over the box of the node's observables
                              by the midpoint rule with the given bins per observable,
                              sum over grid points of shape x cell volume
  density f(x) = shape(root)(x) / norm(root)
  NLL(theta)   = - sum_i log f(x_i; theta)      (non-extended, unweighted)

The gradient is PyTorch autograd of this definition.
"""
import torch

from . import pdfs

_LEAF_PARAMS = {"gauss": 2, "expo": 1, "poly2": 2, "argus": 3}


class TreeModel:
    """A spec's sum/product expression tree (see synth/specs.py for the spec format)."""

    def __init__(self, spec):
        self.spec = spec
        self.obs = {name: (i, float(lo), float(hi)) for i, (name, lo, hi) in enumerate(spec["observables"])}
        self.pidx = {p[0]: i for i, p in enumerate(spec["params"])}
        self.tree = spec["pdf"]
        self.norm_spec = spec["norm"]
        if self.tree[0] == "coherent":
            raise ValueError("amplitude models are handled by oracle.dalitz")

    # -- structure ---------------------------------------------------------------------
    def observables_of(self, node):
        op = node[0]
        if op in _LEAF_PARAMS:
            return {node[1]}
        kids = node[1] if op == "prod" else node[2]
        out = set()
        for k in kids:
            out |= self.observables_of(k)
        return out

    # -- shapes --------------------------------------------------------------------------
    def shape(self, node, X, th, cache):
        op = node[0]
        P = lambda name: th[self.pidx[name]]  # noqa: E731
        if op == "gauss":
            return pdfs.gauss_shape(X[node[1]], P(node[2]), P(node[3]))
        if op == "expo":
            return pdfs.expo_shape(X[node[1]], P(node[2]))
        if op == "poly2":
            return pdfs.poly2_shape(X[node[1]], P(node[2]), P(node[3]))
        if op == "argus":
            return pdfs.argus_shape(X[node[1]], P(node[2]), P(node[3]), P(node[4]))
        if op == "prod":
            out = None
            for k in node[1]:
                v = self.shape(k, X, th, cache)
                out = v if out is None else out * v
            return out
        if op == "add":
            fracs, kids = node[1], node[2]
            assert len(fracs) == len(kids) - 1
            total = None
            rest = 1.0
            for j, k in enumerate(kids):
                if j < len(fracs):
                    w = P(fracs[j])
                    rest = rest - w
                else:
                    w = rest
                term = w * self.shape(k, X, th, cache) / self.norm(k, th, cache)
                total = term if total is None else total + term
            return total
        raise ValueError(f"unknown node {op}")

    # -- normalisation -----------------------------------------------------------------------
    def norm(self, node, th, cache):
        key = id(node)
        if key in cache:
            return cache[key]
        op = node[0]
        kind = self.norm_spec[0]
        if op == "add":
            val = torch.ones((), dtype=torch.float64)
        elif kind == "analytic":
            val = self._analytic_norm(node, th, cache)
        elif kind == "grid":
            val = self.grid_integral(node, th, self.norm_spec[1], cache)
        else:
            raise ValueError(f"unknown normalisation {kind}")
        cache[key] = val
        return val

    def _analytic_norm(self, node, th, cache):
        op = node[0]
        P = lambda name: th[self.pidx[name]]  # noqa: E731
        if op == "prod":
            out = torch.ones((), dtype=torch.float64)
            for k in node[1]:
                out = out * self.norm(k, th, cache)
            return out
        _, lo, hi = self.obs[node[1]]
        if op == "gauss":
            return pdfs.gauss_integral(lo, hi, P(node[2]), P(node[3]))
        if op == "expo":
            return pdfs.expo_integral(lo, hi, P(node[2]))
        if op == "poly2":
            return pdfs.poly2_integral(lo, hi, P(node[2]), P(node[3]))
        raise ValueError(f"{op} has no closed-form normalisation; use grid normalisation")

    def grid_points(self, names, bins):
        """Midpoint grid over the box of the named observables: (dict of columns, cell volume)."""
        axes, vol = [], 1.0
        for nm in names:
            i, lo, hi = self.obs[nm]
            n = int(bins[i])
            h = (hi - lo) / n
            axes.append(lo + (torch.arange(n, dtype=torch.float64) + 0.5) * h)
            vol *= h
        mesh = torch.meshgrid(*axes, indexing="ij")
        return {nm: g.reshape(-1) for nm, g in zip(names, mesh)}, vol

    def grid_integral(self, node, th, bins, cache):
        names = sorted(self.observables_of(node), key=lambda n: self.obs[n][0])
        X, vol = self.grid_points(names, bins)
        return self.shape(node, X, th, cache).sum() * vol

    # -- density and likelihood ------------------------------------------------------------
    def density(self, cols, theta):
        th = torch.as_tensor(theta, dtype=torch.float64)
        X = {k: torch.as_tensor(v, dtype=torch.float64) for k, v in cols.items()}
        cache = {}
        return self.shape(self.tree, X, th, cache) / self.norm(self.tree, th, cache)

    def nll(self, cols, theta, weights=None):
        """-sum_i w_i log f(x_i): unweighted events, or a binned dataset given as bin centres
        with their counts as weights (the multinomial likelihood of the bin contents with f
        at the bin centres; the bin volume is a theta-independent constant and is dropped)."""
        with torch.no_grad():
            lf = torch.log(self.density(cols, theta))
            if weights is not None:
                lf = lf * torch.as_tensor(weights, dtype=torch.float64)
            return float(-lf.sum())

    def nll_grad(self, cols, theta, weights=None):
        th = torch.tensor([float(t) for t in theta], dtype=torch.float64, requires_grad=True)
        X = {k: torch.as_tensor(v, dtype=torch.float64) for k, v in cols.items()}
        cache = {}
        f = self.shape(self.tree, X, th, cache) / self.norm(self.tree, th, cache)
        lf = torch.log(f)
        if weights is not None:
            lf = lf * torch.as_tensor(weights, dtype=torch.float64)
        nll = -lf.sum()
        (g,) = torch.autograd.grad(nll, th)
        return float(nll.detach()), g.numpy().copy()

    def component_norms(self, theta):
        """Norms of the ADD children (or of the root when it is not an ADD), in tree order."""
        th = torch.as_tensor(theta, dtype=torch.float64)
        cache = {}
        root = self.tree
        nodes = root[2] if root[0] == "add" else [root]
        with torch.no_grad():
            return [float(self.norm(k, th, cache)) for k in nodes]


def fd_grad(fn, theta, steps):
    """Central finite differences of a scalar function."""
    theta = [float(t) for t in theta]
    g = []
    for i, h in enumerate(steps):
        tp = list(theta)
        tm = list(theta)
        tp[i] += h
        tm[i] -= h
        g.append((fn(tp) - fn(tm)) / (2.0 * h))
    return g

