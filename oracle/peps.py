"""O3: FP64 PEPS builder and exact contractor -- test infrastructure only.

Follows the paper step by step, in plain NumPy (complex128):

* PEPS equation (main text): the state is a product of rank-5 site tensors
  [A_n^sigma]_{l,r,u,d}, one per qubit, summed over shared auxiliary legs.
  Here A[q] is an ndarray with axes (sigma, l, r, u, d).  The initial product
  state |0...0> has every auxiliary leg of dimension 1, A^0 = 1, A^1 = 0.
* Single-qubit gate absorption (main-text "onebody" equation):
  A'^tau = sum_sigma U^tau_sigma A^sigma; the tensor keeps its size.
* Two-qubit gate absorption (main-text "factorize", "twoqubita/b"): the gate
  O is split as sum_s U_s (x) V_s; U is absorbed into site n and V into site
  m, and the new index s is bundled into the shared leg on both sides, so that
  leg grows by the factor chi_o (2 for CZ).  For CZ the split is the exact
  projector form CZ = P_0 (x) I + P_1 (x) Z (the singular values of CZ are
  degenerate, so its SVD split is not unique; any split gives the same
  amplitudes, which the tests check with an SVD split).  Bundling convention:
  new leg index = old * chi_o + s on both sites; U goes on the site with the
  lower index q = r*C + c.
* Projection on a bitstring (main-text "overlap" equation): E_q = A_q^{tau_q}.
* Exact contraction (supplementary equations for the exact overlap, generic
  scheme): absorb the projected tensors one site at a time into a running
  tensor, row by row from the top and left to right inside a row ("row"
  sweep, the paper's order), or column by column from the left and top to
  bottom inside a column ("column" sweep, the same scheme transposed, which
  the paper allows when the lattice is wider than tall).  Each absorption is
  one np.tensordot over the legs the running tensor shares with the site.

* Square partition (supplementary, Fig. S2(b) and (c) and the "spacesquare*"
  / "timesquare*" equations): the lattice is split into four parts (four
  quarters for even sides; for an odd side 2m+1 an (m+1) x m, an
  (m+1) x (m+1) part holding the centre site, an m x (m+1) and an m x m
  part); each part's projected sites are contracted into one tensor (F_ul,
  F_ur, F_bl, F_br) whose open legs are the edges it shares with the other
  parts; then F_ul is contracted with F_ur and F_bl with F_br, and the two
  results with each other.

* Marginals (the main text's remark on measuring a subset of qubits):
  P(x_S) = <psi| Pi_S |psi> is the same network with every site replaced by
  its double layer D_q = sum_sigma A_q^sigma (x) conj(A_q^sigma), sigma fixed
  to x_q on measured sites and summed over {0, 1} on the others; every bond
  becomes the pair (ket index, bra index).

Slicing (the paper's "cut" technique, named as future work in its
conclusions): fixing the Schmidt index s of chosen CZ gates replaces that
gate by its single term U_s (x) V_s with no bond growth; the amplitude is the
sum over all fixed values.
"""
from __future__ import annotations

import numpy as np

# Axes of a site tensor.
SIGMA, L, R_, U_, D = 0, 1, 2, 3, 4


def cz_projector_split():
    """U[tau, sigma, s], V[s, tau, sigma] with CZ = sum_s U_s (x) V_s."""
    U = np.zeros((2, 2, 2), dtype=np.complex128)
    V = np.zeros((2, 2, 2), dtype=np.complex128)
    for s in range(2):
        U[s, s, s] = 1.0                        # P_s = |s><s|
        V[s, 0, 0] = 1.0                        # Z^s
        V[s, 1, 1] = -1.0 if s == 1 else 1.0
    return U, V


def cz_matrix():
    """CZ as O[tau_n, tau_m, sigma_n, sigma_m]."""
    O = np.zeros((2, 2, 2, 2), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            O[a, b, a, b] = -1.0 if (a == 1 and b == 1) else 1.0
    return O


def svd_split(O: np.ndarray, tol: float = 1e-12):
    """Operator-Schmidt split of a two-qubit gate O[tau_n, tau_m, sigma_n,
    sigma_m] by SVD, singular values absorbed into U (main-text "factorize").
    Returns U[tau_n, sigma_n, s], V[s, tau_m, sigma_m]."""
    M = np.transpose(O, (0, 2, 1, 3)).reshape(4, 4)   # rows (tau_n sigma_n)
    W, S, Vh = np.linalg.svd(M)
    k = int(np.sum(S > tol * S[0]))
    U = (W[:, :k] * S[:k]).reshape(2, 2, k)
    V = Vh[:k, :].reshape(k, 2, 2)
    return U, V


class PEPS:
    """Untruncated PEPS of an R x C lattice, FP64."""

    def __init__(self, R: int, C: int):
        self.R, self.C = R, C
        self.A = []
        for _ in range(R * C):
            t = np.zeros((2, 1, 1, 1, 1), dtype=np.complex128)
            t[0, 0, 0, 0, 0] = 1.0
            self.A.append(t)

    # -- gates -------------------------------------------------------------
    def apply_1q(self, q: int, U: np.ndarray) -> None:
        self.A[q] = np.tensordot(np.asarray(U, dtype=np.complex128), self.A[q], axes=([1], [0]))

    def _shared_axes(self, q0: int, q1: int):
        """(axis on q0, axis on q1) of the bond between neighbours q0 < q1."""
        C = self.C
        r0, c0 = divmod(q0, C)
        r1, c1 = divmod(q1, C)
        if r0 == r1 and c1 == c0 + 1:
            return R_, L
        if c0 == c1 and r1 == r0 + 1:
            return D, U_
        raise ValueError(f"qubits {q0},{q1} are not lattice neighbours")

    def apply_2q_split(self, q0: int, q1: int, U: np.ndarray, V: np.ndarray) -> None:
        """Absorb sum_s U_s (x) V_s: U[tau,sigma,s] on q0, V[s,tau,sigma] on
        q1 (q0 < q1); bundle s into the shared leg as old*chi_o + s."""
        ax0, ax1 = self._shared_axes(q0, q1)
        chi_o = U.shape[2]
        # site q0: A'[tau, l, r, u, d, s] = sum_sigma U[tau, sigma, s] A[sigma, l, r, u, d]
        a0 = np.einsum("tos,olrud->tlruds", U, self.A[q0])
        a0 = np.moveaxis(a0, 5, ax0 + 1)       # s directly after the bundled leg
        sh = list(self.A[q0].shape)
        sh[ax0] *= chi_o
        self.A[q0] = a0.reshape(sh)
        # site q1: A'[tau, l, r, u, d, s] = sum_sigma V[s, tau, sigma] A[sigma, l, r, u, d]
        a1 = np.einsum("sto,olrud->tlruds", V, self.A[q1])
        a1 = np.moveaxis(a1, 5, ax1 + 1)
        sh = list(self.A[q1].shape)
        sh[ax1] *= chi_o
        self.A[q1] = a1.reshape(sh)

    def apply_2q_fixed(self, q0: int, q1: int, U: np.ndarray, V: np.ndarray, s: int) -> None:
        """Absorb the single Schmidt term U_s (x) V_s (a sliced gate)."""
        self._shared_axes(q0, q1)
        self.A[q0] = np.tensordot(U[:, :, s], self.A[q0], axes=([1], [0]))
        self.A[q1] = np.tensordot(V[s], self.A[q1], axes=([1], [0]))

    def apply_2q(self, q0: int, q1: int, G: np.ndarray) -> None:
        """A general two-qubit gate G[(t0 t1), (s0 s1)] (qubit q0 first) by its
        operator-Schmidt split (main-text "factorize": SVD, singular values
        absorbed into U); U goes on the lower-indexed site."""
        G4 = np.asarray(G, dtype=np.complex128).reshape(2, 2, 2, 2)
        if q0 > q1:
            q0, q1 = q1, q0
            G4 = np.transpose(G4, (1, 0, 3, 2))
        U, V = svd_split(G4)
        self.apply_2q_split(q0, q1, U, V)

    def apply_cz(self, q0: int, q1: int, split: str = "projector") -> None:
        a, b = min(q0, q1), max(q0, q1)
        if split == "projector":
            U, V = cz_projector_split()
        elif split == "svd":
            U, V = svd_split(cz_matrix())
        else:
            raise ValueError(split)
        self.apply_2q_split(a, b, U, V)

    # -- queries -----------------------------------------------------------
    def bond_dim(self, q0: int, q1: int) -> int:
        a, b = min(q0, q1), max(q0, q1)
        ax0, ax1 = self._shared_axes(a, b)
        d0, d1 = self.A[a].shape[ax0], self.A[b].shape[ax1]
        assert d0 == d1
        return d0

    def project(self, x: int):
        """E_q = A_q^{tau_q} with tau_q = bit q of x (rank-4, axes l,r,u,d)."""
        return [self.A[q][(int(x) >> q) & 1] for q in range(self.R * self.C)]


def build(R: int, C: int, gates, split: str = "projector", sliced=None, slice_id: int = 0) -> PEPS:
    """Evolve |0...0> through the gate list.  `sliced` is a sequence of CZ
    ordinals (0 = first CZ of the list); bit j of slice_id fixes the Schmidt
    index s of CZ number sliced[j]."""
    p = PEPS(R, C)
    fixed = {}
    if sliced is not None:
        for j, k in enumerate(sliced):
            fixed[int(k)] = (slice_id >> j) & 1
    k = 0
    for g in gates:
        if g.kind == "1q":
            p.apply_1q(g.qubits[0], g.U)
        elif g.kind == "cz":
            if k in fixed:
                U, V = cz_projector_split()
                p.apply_2q_fixed(g.qubits[0], g.qubits[1], U, V, fixed[k])
            else:
                p.apply_cz(g.qubits[0], g.qubits[1], split)
            k += 1
        elif g.kind == "2q":
            p.apply_2q(g.qubits[0], g.qubits[1], g.U)
        else:
            raise ValueError(g.kind)
    return p


# ---------------------------------------------------------------------------
# Exact contraction
# ---------------------------------------------------------------------------

def _leg_labels(R: int, C: int, q: int):
    """Labels of the (l, r, u, d) legs of site q: interior legs are named by
    their edge, boundary legs (dimension 1) get a label of their own."""
    r, c = divmod(q, C)
    lab_l = ("h", r, c - 1) if c > 0 else ("bl", r, c)
    lab_r = ("h", r, c) if c < C - 1 else ("br", r, c)
    lab_u = ("v", r - 1, c) if r > 0 else ("bu", r, c)
    lab_d = ("v", r, c) if r < R - 1 else ("bd", r, c)
    return [lab_l, lab_r, lab_u, lab_d]


def sweep_order(R: int, C: int, sweep: str = "column"):
    if sweep == "column":
        return [r * C + c for c in range(C) for r in range(R)]
    if sweep == "row":
        return [r * C + c for r in range(R) for c in range(C)]
    raise ValueError(sweep)


def absorb(G, labels, E_q, q, R, C):
    """One site absorption: contract the running tensor G (legs `labels`) with
    E_q over every leg they share; the result keeps G's open legs followed by
    E_q's open legs."""
    tl = _leg_labels(R, C, q)
    shared = [lab for lab in tl if lab in labels]
    ga = [labels.index(s) for s in shared]
    ta = [tl.index(s) for s in shared]
    G = np.tensordot(G, E_q, axes=(ga, ta))
    labels = [lab for lab in labels if lab not in shared] + [lab for lab in tl if lab not in shared]
    return G, labels


def contract(E, R: int, C: int, sweep: str = "column", state=None, sites=None):
    """Absorb the sites `sites` (default: all, in sweep order) into `state`
    (default: the scalar 1).  Returns (G, labels)."""
    if state is None:
        G, labels = np.ones((), dtype=np.complex128), []
    else:
        G, labels = state
    if sites is None:
        sites = sweep_order(R, C, sweep)
    for q in sites:
        G, labels = absorb(G, labels, E[q], q, R, C)
    return G, labels


def amplitude(peps: PEPS, x: int, sweep: str = "column") -> complex:
    E = peps.project(x)
    G, _ = contract(E, peps.R, peps.C, sweep)
    assert G.size == 1
    return complex(G.reshape(-1)[0])


def amplitudes(peps: PEPS, bitstrings, sweep: str = "column") -> np.ndarray:
    return np.array([amplitude(peps, int(x), sweep) for x in bitstrings], dtype=np.complex128)


def amplitudes_with_prefix(peps: PEPS, bitstrings, prefix_cols: int) -> np.ndarray:
    """Column sweep in which the running tensor after the first `prefix_cols`
    columns is computed once for every distinct setting of those columns' bits
    and then finished for each bitstring."""
    R, C = peps.R, peps.C
    order = sweep_order(R, C, "column")
    pre_sites = [q for q in order if q % C < prefix_cols]
    post_sites = [q for q in order if q % C >= prefix_cols]
    pre_mask = 0
    for q in pre_sites:
        pre_mask |= 1 << q
    cache = {}
    out = np.zeros(len(bitstrings), dtype=np.complex128)
    for i, x in enumerate(bitstrings):
        x = int(x)
        key = x & pre_mask
        E = peps.project(x)
        if key not in cache:
            cache.clear()
            cache[key] = contract(E, R, C, "column", sites=pre_sites)
        G, _ = contract(E, R, C, "column", state=cache[key], sites=post_sites)
        out[i] = complex(G.reshape(-1)[0])
    return out


def double_layer(peps: PEPS, x: int, mask: int):
    """The double-layer site tensors of P(x_S): D_q[(l,l'),(r,r'),(u,u'),(d,d')]
    = sum_sigma A^sigma[l,r,u,d] conj(A^sigma[l',r',u',d']), sigma = bit q of x
    if bit q of mask is set, else summed over 0 and 1.  The pair index is
    ket * dim + bra."""
    out = []
    for q in range(peps.R * peps.C):
        A = peps.A[q]
        sig = [(int(x) >> q) & 1] if (mask >> q) & 1 else [0, 1]
        D = sum(np.einsum("lrud,LRUD->lLrRuUdD", A[s], np.conj(A[s])) for s in sig)
        dl, dr, du, dd = A.shape[1:]
        out.append(D.reshape(dl * dl, dr * dr, du * du, dd * dd))
    return out


def marginal(peps: PEPS, x: int, mask: int, sweep: str = "column") -> float:
    """P(x_S) by contracting the double-layer network (real up to rounding)."""
    G, _ = contract(double_layer(peps, x, mask), peps.R, peps.C, sweep)
    return float(G.reshape(-1)[0].real)


def marginals(peps: PEPS, bitstrings, mask: int) -> np.ndarray:
    return np.array([marginal(peps, int(x), mask) for x in bitstrings])


def quadrant_sites(R: int, C: int):
    """The four parts of the square partition: {"ul", "ur", "bl", "br"} ->
    their sites in contraction order.  Even R and C (supplementary Fig.
    S2(b)): four R/2 x C/2 quarters.  Odd square side 2m+1 (Fig. S2(c)):
    ul = rows 0..m x cols 0..m-1 ((m+1) x m), ur = rows 0..m x cols m..2m
    ((m+1) x (m+1), holding the centre site), bl = rows m+1..2m x cols 0..m
    (m x (m+1)) and br = rows m+1..2m x cols m+1..2m (m x m).  Every part is
    contracted row by row starting from its corner of the lattice, so the
    open legs toward the other parts appear last."""
    if R % 2 == 0 and C % 2 == 0:
        h, w = R // 2, C // 2
        parts = (("ul", range(0, h), range(0, w)),
                 ("ur", range(0, h), range(C - 1, w - 1, -1)),
                 ("bl", range(R - 1, h - 1, -1), range(0, w)),
                 ("br", range(R - 1, h - 1, -1), range(C - 1, w - 1, -1)))
    elif R == C and R % 2 == 1 and R >= 3:
        m = R // 2
        parts = (("ul", range(0, m + 1), range(0, m)),
                 ("ur", range(0, m + 1), range(C - 1, m - 1, -1)),
                 ("bl", range(R - 1, m, -1), range(0, m + 1)),
                 ("br", range(R - 1, m, -1), range(C - 1, m, -1)))
    else:
        raise ValueError("the square partition needs even sides or an odd square")
    return {name: [r * C + c for r in rows for c in cols] for name, rows, cols in parts}


def merge(a, b):
    """Contract two labelled tensors (G, labels) over every label they share."""
    (ga, la), (gb, lb) = a, b
    shared = [lab for lab in la if lab in lb]
    G = np.tensordot(ga, gb, axes=([la.index(s) for s in shared], [lb.index(s) for s in shared]))
    return G, [lab for lab in la if lab not in shared] + [lab for lab in lb if lab not in shared]


def contract_quadrants(E, R: int, C: int) -> complex:
    """The network of site tensors E by the square partition of Fig. S2(b):
    the four quarter tensors, then upper-left with upper-right and
    bottom-left with bottom-right, then the two halves."""
    F = {name: contract(E, R, C, sites=sites) for name, sites in quadrant_sites(R, C).items()}
    upper = merge(F["ul"], F["ur"])
    lower = merge(F["bl"], F["br"])
    G, _ = merge(upper, lower)
    assert G.size == 1
    return complex(G.reshape(-1)[0])


def amplitude_quadrant(peps: PEPS, x: int) -> complex:
    return contract_quadrants(peps.project(x), peps.R, peps.C)


def marginal_quadrant(peps: PEPS, x: int, mask: int) -> float:
    """P(x_S) by the square partition of the double-layer network."""
    return contract_quadrants(double_layer(peps, x, mask), peps.R, peps.C).real


def amplitudes_quadrant(peps: PEPS, bitstrings) -> np.ndarray:
    return np.array([amplitude_quadrant(peps, int(x)) for x in bitstrings], dtype=np.complex128)


def quadrant_contraction_cmacs(R: int, C: int, dims) -> dict:
    """Complex multiply-adds of the square partition, counted directly from
    the bond dimensions dims[(q0, q1)] (no formula): every contraction of two
    tensors costs prod(legs of the first) x prod(legs of the second not
    contracted).  Returns {"quarters": .., "merges": .., "largest": entries}."""
    def legdims(q):
        r, c = divmod(q, C)
        out = []
        for lab in _leg_labels(R, C, q):
            if lab[0] == "h":
                a = lab[1] * C + lab[2]
                out.append((lab, dims[(a, a + 1)]))
            elif lab[0] == "v":
                a = lab[1] * C + lab[2]
                out.append((lab, dims[(a, a + C)]))
            else:
                out.append((lab, 1))
        return out

    def cost(la, lb):
        shared = [k for k in la if k in lb]
        c = 1
        for k in la:
            c *= la[k]
        for k in lb:
            if k not in shared:
                c *= lb[k]
        out = {k: v for k, v in la.items() if k not in shared}
        out.update({k: v for k, v in lb.items() if k not in shared})
        return c, out

    quarters, largest, F = 0, 1, {}
    for name, sites in quadrant_sites(R, C).items():
        G = {}
        for q in sites:
            c, G = cost(G, dict(legdims(q)))
            quarters += c
            largest = max(largest, int(np.prod(list(G.values()))))
        F[name] = G
    merges = 0
    c, up = cost(F["ul"], F["ur"])
    merges += c
    c, lo = cost(F["bl"], F["br"])
    merges += c
    largest = max(largest, int(np.prod(list(up.values()))), int(np.prod(list(lo.values()))))
    c, _ = cost(up, lo)
    merges += c
    return {"quarters": quarters, "merges": merges, "largest": largest}


def column_contraction_cmacs(R: int, C: int, dims) -> int:
    """Complex multiply-adds of the column sweep, from the bond dimensions
    dims[(q0, q1)], counted as prod(all legs of G before absorption) x
    prod(open legs of the site) for every step (a direct count, no formula)."""
    order = sweep_order(R, C, "column")
    legdim = {}
    total = 0
    labels = []
    for q in order:
        tl = _leg_labels(R, C, q)
        sizes = []
        for lab in tl:
            if lab[0] in ("h", "v"):
                if lab[0] == "h":
                    a = lab[1] * C + lab[2]
                    b = a + 1
                else:
                    a = lab[1] * C + lab[2]
                    b = a + C
                sizes.append(dims[(a, b)])
            else:
                sizes.append(1)
        shared = [lab for lab in tl if lab in labels]
        g_size = 1
        for lab in labels:
            g_size *= legdim[lab]
        open_size = 1
        for lab, s in zip(tl, sizes):
            legdim[lab] = s
            if lab not in shared:
                open_size *= s
        total += g_size * open_size
        labels = [lab for lab in labels if lab not in shared] + [lab for lab in tl if lab not in shared]
    return total
