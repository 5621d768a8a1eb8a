"""Seeded synthetic inputs shared by the CUDA engine's tests/bench and by the CPU oracle.

This module defines *inputs* only: lattices and their site orderings, Hamiltonians written
as sums of operator strings, the matrix-product-operator (MPO) encoding of such a sum, and
seeded random U(1) block-sparse matrix product states.  It performs none of the DMRG
method's arithmetic (no eigen-solver, no SVD, no environment contraction).

Models follow the paper's workloads: the spin-1/2 Heisenberg model on chains and on square
and triangular cylinders (Sec. III, Fig. 1: 24x8 square cylinder; Sec. III.B: triangular
cylinders, H = J sum S_i.S_j), the pure Q2 model written as products of two bond operators
(Sec. III.A, Eq. q2), plus the transverse-field Ising and AKLT chains used as closed-form pins.

Conventions
-----------
* Local basis charges are 2*S^z integers.  Spin-1/2 basis order is (up, down) -> (+1, -1);
  spin-1 order is (+1, 0, -1) -> (+2, 0, -2).  Models without U(1) symmetry (transverse-field
  Ising) use all-zero charges, so every bond has a single sector (dense DMRG).
* An MPO tensor W_j has shape [D_j, d, d, D_{j+1}] with W_j[w, s, s', w'] = <s|op|s'>.
  Every MPO bond index w carries a flux f(w): the total charge raised by the operators
  already placed to its left.  W_j[w, s, s', w'] != 0 implies q(s) - q(s') = f(w') - f(w).
* Channel 0 of every inner bond is IDLE (identity so far), the last is DONE (a full term
  already placed); D_0 = D_L = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------------------
# Local Hilbert spaces
# ----------------------------------------------------------------------------------------


@dataclass(frozen=True)
class SiteType:
    name: str
    qn: tuple          # 2*S^z (or 0) of each local basis state
    ops: dict = field(hash=False, compare=False)

    @property
    def d(self) -> int:
        return len(self.qn)

    def op(self, name: str) -> np.ndarray:
        """Operator by name; 'A*B' is the single-site product A @ B."""
        mats = [self.ops[n] for n in name.split("*")]
        out = mats[0]
        for m in mats[1:]:
            out = out @ m
        return out

    def charge(self, name: str) -> int:
        """Charge raised by operator `name` (q(s) - q(s') on its nonzero elements)."""
        m = self.op(name)
        qs = None
        for s in range(self.d):
            for sp in range(self.d):
                if abs(m[s, sp]) > 0:
                    c = self.qn[s] - self.qn[sp]
                    if qs is None:
                        qs = c
                    elif qs != c:
                        raise ValueError(f"operator {name} has no definite charge")
        return 0 if qs is None else qs


def spin_half() -> SiteType:
    sz = np.diag([0.5, -0.5])
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    return SiteType("spin_half", (1, -1), {"Id": np.eye(2), "Sz": sz, "Sp": sp, "Sm": sp.T.copy()})


def spin_half_pauli() -> SiteType:
    """Spin-1/2 in the sigma^z basis without U(1) labels (for the transverse-field Ising chain)."""
    x = np.array([[0.0, 1.0], [1.0, 0.0]])
    z = np.diag([1.0, -1.0])
    return SiteType("spin_half_pauli", (0, 0), {"Id": np.eye(2), "X": x, "Z": z})


def spin_one() -> SiteType:
    sz = np.diag([1.0, 0.0, -1.0])
    sp = np.zeros((3, 3))
    sp[0, 1] = math.sqrt(2.0)
    sp[1, 2] = math.sqrt(2.0)
    return SiteType("spin_one", (2, 0, -2), {"Id": np.eye(3), "Sz": sz, "Sp": sp, "Sm": sp.T.copy()})


# ----------------------------------------------------------------------------------------
# Lattices (bond lists in the 1D MPS ordering)
# ----------------------------------------------------------------------------------------


def chain_bonds(L: int):
    return [(i, i + 1) for i in range(L - 1)]


def snake_index(x: int, y: int, Ly: int) -> int:
    """Snake ordering of a cylinder: columns x in order, y reversed on odd columns."""
    return x * Ly + (y if x % 2 == 0 else Ly - 1 - y)


def square_cylinder_bonds(Lx: int, Ly: int):
    """Nearest-neighbour bonds of an Lx x Ly square cylinder, periodic in y, open in x."""
    bonds = set()
    for x in range(Lx):
        for y in range(Ly):
            i = snake_index(x, y, Ly)
            if x + 1 < Lx:
                bonds.add(tuple(sorted((i, snake_index(x + 1, y, Ly)))))
            if Ly > 2 or y + 1 < Ly:
                j = snake_index(x, (y + 1) % Ly, Ly)
                if i != j:
                    bonds.add(tuple(sorted((i, j))))
    return sorted(bonds)


def triangular_cylinder_bonds(Lx: int, Ly: int):
    """Triangular cylinder: square-cylinder bonds plus the (x,y)-(x+1,y-1) diagonal."""
    bonds = set(square_cylinder_bonds(Lx, Ly))
    for x in range(Lx - 1):
        for y in range(Ly):
            i = snake_index(x, y, Ly)
            j = snake_index(x + 1, (y - 1) % Ly, Ly)
            bonds.add(tuple(sorted((i, j))))
    return sorted(bonds)


def square_plaquettes(Lx: int, Ly: int):
    """Elementary plaquettes of the square cylinder as corner tuples (r, r+x, r+y, r+x+y)."""
    plaq = []
    for x in range(Lx - 1):
        for y in range(Ly if Ly > 2 else Ly - 1):
            a = snake_index(x, y, Ly)
            b = snake_index(x + 1, y, Ly)
            c = snake_index(x, (y + 1) % Ly, Ly)
            e = snake_index(x + 1, (y + 1) % Ly, Ly)
            plaq.append((a, b, c, e))
    return plaq


# ----------------------------------------------------------------------------------------
# Hamiltonians as operator strings: list of (coef, ((site, opname), ...)), sites ascending
# ----------------------------------------------------------------------------------------


def _string(coef, *site_ops):
    """Normalise one term: merge repeated sites into single-site products, sort by site."""
    by_site = {}
    for s, o in site_ops:
        by_site.setdefault(s, []).append(o)
    ops = tuple((s, "*".join(by_site[s])) for s in sorted(by_site))
    return (float(coef), ops)


def heisenberg_terms(bonds, J=1.0):
    """H = sum_<ij> J_ij S_i.S_j = J (Sz Sz + (S+ S- + S- S+)/2).  `J` scalar or per-bond list."""
    Js = [J] * len(bonds) if np.isscalar(J) else list(J)
    terms = []
    for (i, j), Jij in zip(bonds, Js):
        terms.append(_string(Jij, (i, "Sz"), (j, "Sz")))
        terms.append(_string(0.5 * Jij, (i, "Sp"), (j, "Sm")))
        terms.append(_string(0.5 * Jij, (i, "Sm"), (j, "Sp")))
    return terms


def field_terms(hz):
    """H = sum_i hz_i S^z_i."""
    return [_string(float(h), (i, "Sz")) for i, h in enumerate(hz)]


def tfim_terms(L, J=1.0, h=1.0):
    """H = -J sum sigma^z_i sigma^z_{i+1} - h sum sigma^x_i (open chain)."""
    terms = [_string(-J, (i, "Z"), (i + 1, "Z")) for i in range(L - 1)]
    terms += [_string(-h, (i, "X")) for i in range(L)]
    return terms


_SDOT = (("Sz", "Sz", 1.0), ("Sp", "Sm", 0.5), ("Sm", "Sp", 0.5))


def aklt_terms(L):
    """H = sum_i [S_i.S_{i+1} + (1/3)(S_i.S_{i+1})^2] for spin 1 (open chain)."""
    terms = []
    for i in range(L - 1):
        for a, b, c in _SDOT:
            terms.append(_string(c, (i, a), (i + 1, b)))
        for a1, b1, c1 in _SDOT:
            for a2, b2, c2 in _SDOT:
                terms.append(_string(c1 * c2 / 3.0, (i, a1), (i, a2), (i + 1, b1), (i + 1, b2)))
    return terms


def jq2_terms(Lx, Ly, J, Q):
    """J-Q2 model: sum_b J_b S_i.S_j - sum_p Q_p [(S_i.S_j - 1/4)(S_k.S_l - 1/4)] over both
    pairs of opposite edges of each plaquette (Eq. q2).  J, Q: per-bond / per-(plaquette,
    orientation) coefficient lists."""
    bonds = square_cylinder_bonds(Lx, Ly)
    terms = heisenberg_terms(bonds, J)
    pairs = []
    for (a, b, c, e) in square_plaquettes(Lx, Ly):
        pairs.append(((a, b), (c, e)))   # two horizontal edges
        pairs.append(((a, c), (b, e)))   # two vertical edges
    for ((i, j), (k, l)), q in zip(pairs, Q):
        # (S_i.S_j - 1/4)(S_k.S_l - 1/4) = (S_i.S_j)(S_k.S_l) - (S_i.S_j)/4 - (S_k.S_l)/4 + 1/16
        for a1, b1, c1 in _SDOT:
            for a2, b2, c2 in _SDOT:
                terms.append(_string(-q * c1 * c2, (i, a1), (j, b1), (k, a2), (l, b2)))
        for a1, b1, c1 in _SDOT:
            terms.append(_string(q * c1 / 4.0, (i, a1), (j, b1)))
            terms.append(_string(q * c1 / 4.0, (k, a1), (l, b1)))
        terms.append(_string(-q / 16.0, (i, "Id")))
    return terms, pairs


# ----------------------------------------------------------------------------------------
# Finite-state-machine MPO from operator strings (prefix channels)
# ----------------------------------------------------------------------------------------


@dataclass
class MPO:
    site: SiteType
    W: list            # W[j]: ndarray [D_j, d, d, D_{j+1}]
    flux: list         # flux[b]: int ndarray [D_b], b = 0..L
    qtot: int = 0

    @property
    def L(self) -> int:
        return len(self.W)

    @property
    def D(self):
        return [len(f) for f in self.flux]


def build_mpo(L: int, site: SiteType, terms, qtot: int = 0) -> MPO:
    """Encode H = sum_t coef_t prod_k op_{t,k}(site_{t,k}) as an MPO whose channels are the
    distinct operator prefixes still waiting for their remaining factors."""
    alive = [set() for _ in range(L + 1)]
    for coef, ops in terms:
        if sum(site.charge(n) for _, n in ops) != 0:
            raise ValueError("Hamiltonian term does not conserve the U(1) charge")
        for k in range(len(ops) - 1):
            pre = ops[: k + 1]
            for b in range(ops[k][0] + 1, ops[k + 1][0] + 1):
                alive[b].add(pre)
    index = []
    flux = []
    for b in range(L + 1):
        order = (["IDLE"] if b < L else []) + sorted(alive[b]) + (["DONE"] if b > 0 else [])
        index.append({key: i for i, key in enumerate(order)})
        flux.append(np.array([0 if isinstance(k, str) else sum(site.charge(n) for _, n in k)
                              for k in order], dtype=np.int64))
    d = site.d
    W = [np.zeros((len(index[j]), d, d, len(index[j + 1]))) for j in range(L)]
    ident = site.op("Id")
    for j in range(L):
        a, b = index[j], index[j + 1]
        for key in ("IDLE", "DONE"):
            if key in a and key in b:
                W[j][a[key], :, :, b[key]] = ident
        for key in alive[j] & alive[j + 1]:
            W[j][a[key], :, :, b[key]] = ident
    placed = set()
    for coef, ops in terms:
        for k, (s, name) in enumerate(ops):
            frm = "IDLE" if k == 0 else ops[:k]
            last = k == len(ops) - 1
            to = "DONE" if last else ops[: k + 1]
            wi, wo = index[s][frm], index[s + 1][to]
            if last:
                W[s][wi, :, :, wo] += coef * site.op(name)
            elif (s, frm, to) not in placed:
                placed.add((s, frm, to))
                W[s][wi, :, :, wo] = site.op(name)
    return MPO(site=site, W=W, flux=flux, qtot=qtot)


# ----------------------------------------------------------------------------------------
# Seeded random U(1) block-sparse MPS
# ----------------------------------------------------------------------------------------


@dataclass
class BlockMPS:
    """bonds[b]: dict charge -> dim (b = 0..L); sites[j]: dict (q_left, s) -> [m_ql, m_qr]."""
    bonds: list
    sites: list


def _reachable(L, qn):
    """counts[b][q] = number of product states of b sites with total charge q."""
    counts = [{0: 1}]
    for _ in range(L):
        nxt = {}
        for q, c in counts[-1].items():
            for s in qn:
                nxt[q + s] = nxt.get(q + s, 0) + c
        counts.append(nxt)
    return counts


def bond_sectors(L, qn, qtot, m, sigma=None):
    """Sector dims for every bond: exact dims capped at about m in total.  With `sigma`, the
    dims follow a Gaussian profile exp(-(q-q0)^2/(2 sigma^2)) around the mean charge, as in
    the Schmidt spectra of ground states (sectors rounding to zero are dropped); otherwise
    they follow the exact sector sizes with at least one state per reachable sector."""
    left = _reachable(L, qn)
    bonds = []
    for b in range(L + 1):
        exact = {}
        for q, c in left[b].items():
            cr = left[L - b].get(qtot - q, 0)
            if cr > 0:
                exact[q] = min(c, cr)
        total = sum(exact.values())
        if total <= m:
            bonds.append(dict(sorted(exact.items())))
            continue
        if sigma is None:
            wts = {q: exact[q] / total for q in exact}
        else:
            q0 = qtot * b / L
            raw = {q: math.exp(-((q - q0) ** 2) / (2.0 * sigma * sigma)) for q in exact}
            z = sum(raw.values())
            wts = {q: raw[q] / z for q in raw}
        dims = {}
        for q in exact:
            k = min(exact[q], int(math.floor(m * wts[q] + 0.5)))
            if sigma is None:
                k = max(k, 1)          # keep every reachable sector alive
            if k > 0:
                dims[q] = k
        bonds.append(dict(sorted(dims.items())))
    return bonds


def random_mps(L, qn, qtot, m, seed, sigma=None) -> BlockMPS:
    """Normal(0,1) entries on every allowed block, drawn from numpy default_rng(seed) in the
    canonical block order (site, left sector ascending, local state ascending)."""
    rng = np.random.default_rng(seed)
    bonds = bond_sectors(L, qn, qtot, m, sigma)
    sites = []
    for j in range(L):
        blocks = {}
        for ql, ml in bonds[j].items():
            for s, qs in enumerate(qn):
                mr = bonds[j + 1].get(ql + qs)
                if mr:
                    blocks[(ql, s)] = rng.standard_normal((ml, mr))
        sites.append(blocks)
    return BlockMPS(bonds=bonds, sites=sites)


# ----------------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------------


def heisenberg_chain(L, J=1.0, spin="half"):
    site = spin_half() if spin == "half" else spin_one()
    return build_mpo(L, site, heisenberg_terms(chain_bonds(L), J))


def heisenberg_square_cylinder(Lx, Ly, J=1.0):
    return build_mpo(Lx * Ly, spin_half(), heisenberg_terms(square_cylinder_bonds(Lx, Ly), J))


def field_square_cylinder(Lx, Ly, seed, width=0.5, J=1.0):
    """Heisenberg square cylinder plus a random longitudinal field sum_i h_i S^z_i, h_i i.i.d.
    U[-width, width] from default_rng(seed): S^z_tot is still conserved (U(1)), but neither the
    SU(2) multiplets nor the spin-flip pairs of Schmidt values are degenerate any more, so a
    truncation cut has no symmetry-enforced ties."""
    h = np.random.default_rng(seed).uniform(-width, width, Lx * Ly)
    terms = heisenberg_terms(square_cylinder_bonds(Lx, Ly), J) + field_terms(h)
    return build_mpo(Lx * Ly, spin_half(), terms)


def heisenberg_triangular_cylinder(Lx, Ly, J=1.0):
    return build_mpo(Lx * Ly, spin_half(), heisenberg_terms(triangular_cylinder_bonds(Lx, Ly), J))


def tfim_chain(L, J=1.0, h=1.0):
    return build_mpo(L, spin_half_pauli(), tfim_terms(L, J, h))


def aklt_chain(L):
    return build_mpo(L, spin_one(), aklt_terms(L))


def jq2_cylinder(Lx, Ly, seed=1, lo=0.5, hi=2.0):
    """J-Q2 cylinder with per-term couplings J_b, Q_p drawn i.i.d. U[lo, hi] from
    numpy default_rng(seed) (bonds first, then plaquette pairs)."""
    rng = np.random.default_rng(seed)
    bonds = square_cylinder_bonds(Lx, Ly)
    nb = len(bonds)
    npairs = 2 * len(square_plaquettes(Lx, Ly))
    J = rng.uniform(lo, hi, nb)
    Q = rng.uniform(lo, hi, npairs)
    terms, _ = jq2_terms(Lx, Ly, J, Q)
    return build_mpo(Lx * Ly, spin_half(), terms), J, Q


# ----------------------------------------------------------------------------------------
# Flat (packed) layouts used at the C ABI boundary
# ----------------------------------------------------------------------------------------


def pack_mpo(mpo: MPO):
    """Concatenate W tensors (row-major [D_j][d][d][D_{j+1}]) and fluxes for the C ABI."""
    W = np.concatenate([w.ravel() for w in mpo.W]).astype(np.float64)
    flux = np.concatenate(mpo.flux).astype(np.int32)
    D = np.array(mpo.D, dtype=np.int32)
    return W, flux, D


def pack_bond(bond: dict):
    q = np.array(list(bond.keys()), dtype=np.int32)
    m = np.array(list(bond.values()), dtype=np.int32)
    return q, m


def pack_site(blocks: dict, bl: dict, br: dict, qn):
    """Blocks of one site tensor in canonical order: left sector ascending, then local
    state ascending; each block row-major [m_left][m_right]."""
    out = []
    for ql in bl:
        for s, qs in enumerate(qn):
            if (ql + qs) in br and (ql, s) in blocks:
                out.append(np.asarray(blocks[(ql, s)], dtype=np.float64).ravel())
    return np.concatenate(out) if out else np.zeros(0)


def unpack_site(flat, bl: dict, br: dict, qn):
    blocks = {}
    off = 0
    for ql, ml in bl.items():
        for s, qs in enumerate(qn):
            mr = br.get(ql + qs)
            if mr:
                blocks[(ql, s)] = np.asarray(flat[off: off + ml * mr]).reshape(ml, mr)
                off += ml * mr
    return blocks


# ----------------------------------------------------------------------------------------
# Seeded random mixed-canonical MPS (benchmark states at large m)
# ----------------------------------------------------------------------------------------


def consistent_sectors(bonds, qn):
    """Shrink sector dims until every sector of bond b is reachable from both neighbours with
    at least as many states (needed for left/right isometries); drops empty sectors."""
    bonds = [dict(b) for b in bonds]
    L = len(bonds) - 1
    changed = True
    while changed:
        changed = False
        for b in range(1, L + 1):
            for q in list(bonds[b]):
                avail = sum(bonds[b - 1].get(q - s, 0) for s in qn)
                if avail < bonds[b][q]:
                    changed = True
                    if avail == 0:
                        del bonds[b][q]
                    else:
                        bonds[b][q] = avail
        for b in range(L - 1, -1, -1):
            for q in list(bonds[b]):
                avail = sum(bonds[b + 1].get(q + s, 0) for s in qn)
                if avail < bonds[b][q]:
                    changed = True
                    if avail == 0:
                        del bonds[b][q]
                    else:
                        bonds[b][q] = avail
    return bonds


def isometric_mps(L, qn, qtot, m, seed, center, sigma=None) -> BlockMPS:
    """Random MPS in mixed-canonical form around `center`: sites < center are random left
    isometries, sites > center random right isometries (QR of Gaussian matrices), the centre
    a normalised Gaussian tensor.  Draws from numpy default_rng(seed), site by site."""
    rng = np.random.default_rng(seed)
    bonds = consistent_sectors(bond_sectors(L, qn, qtot, m, sigma), qn)
    sites = []
    for j in range(L):
        bl, br = bonds[j], bonds[j + 1]
        blocks = {}
        if j < center:
            for qr, mr in br.items():
                rows = [(ql, s) for ql in bl for s, qs in enumerate(qn) if ql + qs == qr]
                n = sum(bl[ql] for ql, _ in rows)
                Q, _ = np.linalg.qr(rng.standard_normal((n, mr)))
                o = 0
                for (ql, s) in rows:
                    blocks[(ql, s)] = Q[o: o + bl[ql], :].copy()
                    o += bl[ql]
        elif j > center:
            for ql, ml in bl.items():
                cols = [(s, ql + qs) for s, qs in enumerate(qn) if (ql + qs) in br]
                n = sum(br[qr] for _, qr in cols)
                Q, _ = np.linalg.qr(rng.standard_normal((n, ml)))
                Bm = Q.T
                o = 0
                for (s, qr) in cols:
                    blocks[(ql, s)] = Bm[:, o: o + br[qr]].copy()
                    o += br[qr]
        else:
            for ql, ml in bl.items():
                for s, qs in enumerate(qn):
                    mr = br.get(ql + qs)
                    if mr:
                        blocks[(ql, s)] = rng.standard_normal((ml, mr))
            nrm = math.sqrt(sum(float(np.sum(b * b)) for b in blocks.values()))
            blocks = {k: v / nrm for k, v in blocks.items()}
        sites.append(blocks)
    return BlockMPS(bonds=bonds, sites=sites)
