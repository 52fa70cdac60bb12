"""Seeded synthetic inputs: QC-LDPC codes, GF(2) encoders and the BPSK/AWGN channel.

This module is shared by the CPU oracle tests and the CUDA path.  It holds none of
the decoding arithmetic: it builds parity-check matrices, codewords and channel
log-likelihood ratios, nothing else.

Code model (Sec. II): an (N, K) binary LDPC code given by its Tanner graph, here
as a quasi-cyclic (QC) base matrix ``B`` (m_b x n_b, entry -1 = all-zero block,
entry s in [0, Z) = the Z x Z identity cyclically shifted by s).  Circulant
convention (the paper is silent; the 5G NR convention is used):
``H[r*Z + i, c*Z + (i + s) % Z] = 1``.

Channel (Sec. V, first paragraph): BPSK (bit 0 -> +1, bit 1 -> -1) over AWGN,
``sigma^2 = 1 / (2 R 10^(EbN0/10))`` with R = K/N, and the channel LLR of the
suppressed Step-1 initialisation of Sec. II-A, ``L = ln Pr(y|0)/Pr(y|1) = 2y/sigma^2``.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

CODES_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "codes")


# ----------------------------------------------------------------------------
# QC code container
# ----------------------------------------------------------------------------
@dataclass
class QCCode:
    """A quasi-cyclic LDPC code: base matrix + lifting size Z."""

    base: np.ndarray  # int32 [mb, nb], -1 = zero block
    Z: int
    name: str = ""
    _H_rows: list | None = field(default=None, repr=False, compare=False)

    def __post_init__(self):
        self.base = np.ascontiguousarray(np.asarray(self.base, dtype=np.int32))
        if self.base.ndim != 2:
            raise ValueError("base matrix must be 2-D")
        if self.Z < 1:
            raise ValueError("Z must be >= 1")
        if ((self.base < -1) | (self.base >= self.Z)).any():
            raise ValueError("base entries must be -1 or in [0, Z)")

    @property
    def mb(self) -> int:
        return int(self.base.shape[0])

    @property
    def nb(self) -> int:
        return int(self.base.shape[1])

    @property
    def N(self) -> int:
        return self.nb * self.Z

    @property
    def M(self) -> int:
        return self.mb * self.Z

    @property
    def nnz_base(self) -> int:
        return int((self.base >= 0).sum())

    @property
    def E(self) -> int:
        return self.nnz_base * self.Z

    def check_rows(self) -> list[np.ndarray]:
        """Variables of every check m = r*Z + i, ascending (= ascending base column)."""
        if self._H_rows is None:
            rows = []
            Z = self.Z
            for r in range(self.mb):
                cols = np.nonzero(self.base[r] >= 0)[0]
                for i in range(Z):
                    rows.append(np.array([c * Z + (i + int(self.base[r, c])) % Z for c in cols],
                                         dtype=np.int64))
            self._H_rows = rows
        return self._H_rows

    def dense_H(self) -> np.ndarray:
        """Dense uint8 parity-check matrix (small codes only)."""
        H = np.zeros((self.M, self.N), dtype=np.uint8)
        for m, vs in enumerate(self.check_rows()):
            H[m, vs] = 1
        return H

    def syndrome(self, bits: np.ndarray) -> np.ndarray:
        """GF(2) syndrome of hard decisions ``bits`` [F, N] (uint8) -> [F, M]."""
        bits = np.asarray(bits, dtype=np.uint8)
        out = np.zeros((bits.shape[0], self.M), dtype=np.uint8)
        for m, vs in enumerate(self.check_rows()):
            out[:, m] = np.bitwise_xor.reduce(bits[:, vs], axis=1)
        return out


def four_cycle_at(base: np.ndarray, Z: int, r: int, c: int, s: int) -> bool:
    """True if shift s at (r, c) closes a length-4 cycle with the existing entries.

    Rows r, r2 and columns c, c2 form a 4-cycle in the lifted graph iff
    s(r,c) - s(r,c2) + s(r2,c2) - s(r2,c) == 0 (mod Z).
    """
    mb, nb = base.shape
    row_r = base[r]
    col_c = base[:, c]
    for c2 in range(nb):
        if c2 == c or row_r[c2] < 0:
            continue
        col_c2 = base[:, c2]
        for r2 in range(mb):
            if r2 == r or col_c[r2] < 0 or col_c2[r2] < 0:
                continue
            if (s - int(row_r[c2]) + int(col_c2[r2]) - int(col_c[r2])) % Z == 0:
                return True
    return False


def _place(base, Z, r, c, rng, tries=200) -> bool:
    for _ in range(tries):
        s = int(rng.integers(Z))
        if not four_cycle_at(base, Z, r, c, s):
            base[r, c] = s
            return True
    return False


def make_dual_diagonal_code(mb: int, nb: int, Z: int, col_weight: int, seed: int,
                            parity: str = "bidiagonal") -> np.ndarray:
    """Rate (nb-mb)/nb code: info columns of fixed weight + a dual-diagonal parity part.

    parity="bidiagonal": parity column of row r is kb + r (shift 0) and row r >= 1 also
    holds column kb + r - 1 (shift 0), so the last column has weight 1.
    parity="hb": the IEEE 802.16e form -- the first parity column kb has weight 3 (rows
    0 and mb - 1 with shift 1, row mb // 2 with shift 0) and columns kb + j, j >= 1, hold
    rows j - 1 and j (shift 0): no parity column of weight 1.
    Info columns get ``col_weight`` distinct random rows with shifts uniform in [0, Z),
    resampled while they close a 4-cycle.  Draw order: info columns ascending, rows sorted.
    """
    rng = np.random.default_rng(seed)
    kb = nb - mb
    for _attempt in range(1000):
        base = -np.ones((mb, nb), dtype=np.int32)
        if parity == "bidiagonal":
            for r in range(mb):
                base[r, kb + r] = 0
                if r >= 1:
                    base[r, kb + r - 1] = 0
        elif parity == "hb":
            base[0, kb] = base[mb - 1, kb] = 1 % Z
            base[mb // 2, kb] = 0
            for j in range(1, mb):
                base[j - 1, kb + j] = 0
                base[j, kb + j] = 0
        else:
            raise ValueError(parity)
        ok = True
        for c in range(kb):
            placed = False
            for _ in range(100):
                rows = np.sort(rng.choice(mb, size=col_weight, replace=False))
                done = []
                for r in rows:
                    if not _place(base, Z, int(r), c, rng):
                        break
                    done.append(int(r))
                if len(done) == col_weight:
                    placed = True
                    break
                for r in done:
                    base[r, c] = -1
            if not placed:
                ok = False
                break
        deg = (base >= 0).sum(axis=1)
        if ok and (deg >= 2).all():
            return base
    raise RuntimeError("code construction failed")


def make_extension_code(mb: int, nb: int, kb: int, core: int, Z: int, density: float,
                        seed: int, min_core: int = 2) -> np.ndarray:
    """Base graph with a dual-diagonal core and weight-1 extension columns.

    Rows 0..core-1 x columns kb..kb+core-1: lower bidiagonal (shift 0).
    Rows r >= core: column kb + r with shift 0 (a weight-1 extension column).
    Every other entry of the info columns 0..kb-1 (all rows) and of the core
    parity columns (extension rows) is present with probability ``density``,
    with a shift uniform in [0, Z) resampled while it closes a 4-cycle.
    Draw order: rows ascending, columns ascending.  Then every info column is
    topped up to ``min_core`` entries in the core rows (random core rows, same
    generator): an info column absent from the core would form, with its
    weight-1 extension parities, codewords of weight 1 + (column weight).
    """
    if nb != kb + mb:
        raise ValueError("nb must equal kb + mb")
    rng = np.random.default_rng(seed)
    base = -np.ones((mb, nb), dtype=np.int32)
    for r in range(core):
        base[r, kb + r] = 0
        if r >= 1:
            base[r, kb + r - 1] = 0
    for r in range(core, mb):
        base[r, kb + r] = 0
    for r in range(mb):
        ncols = kb if r < core else kb + core
        for c in range(ncols):
            if base[r, c] >= 0:
                continue
            if rng.random() < density:
                _place(base, Z, r, c, rng)
    # repair: every row needs degree >= 2 and every info column weight >= 1
    for r in range(mb):
        while (base[r] >= 0).sum() < 2:
            c = int(rng.integers(kb))
            if base[r, c] < 0:
                _place(base, Z, r, c, rng)
    for c in range(kb):
        while (base[:, c] >= 0).sum() < 1:
            r = int(rng.integers(mb))
            _place(base, Z, r, c, rng)
    for c in range(kb):
        while (base[:core, c] >= 0).sum() < min(min_core, core):
            r = int(rng.integers(core))
            if base[r, c] < 0:
                _place(base, Z, r, c, rng)
    return base


# ----------------------------------------------------------------------------
# committed base matrices
# ----------------------------------------------------------------------------
def save_base(path: str, base: np.ndarray, Z: int, comment: str) -> None:
    mb, nb = base.shape
    with open(path, "w") as f:
        for line in comment.strip().splitlines():
            f.write("# " + line + "\n")
        f.write(f"{mb} {nb} {Z}\n")
        for r in range(mb):
            f.write(" ".join(f"{int(v):d}" for v in base[r]) + "\n")


def load_base(path: str) -> tuple[np.ndarray, int]:
    vals = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            vals.append([int(t) for t in line.split()])
    mb, nb, Z = vals[0]
    base = np.array(vals[1:], dtype=np.int32)
    if base.shape != (mb, nb):
        raise ValueError(f"{path}: expected {mb}x{nb} base matrix, got {base.shape}")
    return base, Z


def load_code(name: str) -> QCCode:
    base, Z = load_base(os.path.join(CODES_DIR, name + ".txt"))
    return QCCode(base, Z, name=name)


def code_576() -> QCCode:
    """12x24 base, Z=24, N=576, rate 1/2, seed 1 (the small parity workload)."""
    return load_code("qc_12x24_z24_seed1")


def code_26112() -> QCCode:
    """46x68 base, Z=384, N=26112, rate 22/68 (the large-batch throughput workload)."""
    return load_code("qc_46x68_z384_seed2")


def code_2304_hb() -> QCCode:
    """12x24, Z=96 (N=2304, rate 1/2), seed 4, with the 802.16e parity part (no weight-1
    column)."""
    return load_code("qc_12x24_z96_seed4_hb")


def code_2304() -> QCCode:
    """12x24 base, Z=96, N=2304, rate 1/2, seed 4."""
    return load_code("qc_12x24_z96_seed4")


def mixed_codes() -> list[QCCode]:
    """The eight codes of the mixed batch: Z = 16 ... 384, rates 1/3 ... 8/9."""
    names = ["mix0_16x24_z16", "mix1_15x25_z32", "mix2_12x24_z64", "mix3_8x24_z96",
             "mix4_6x24_z128", "mix5_4x24_z192", "mix6_3x27_z256", "mix7_12x24_z384"]
    return [load_code(n) for n in names]


# ----------------------------------------------------------------------------
# progressive edge growth (PEG) codes, the code family of the paper's Sec. V
# ----------------------------------------------------------------------------
def peg_graph(var_degrees, m: int, seed: int) -> list[list[int]]:
    """Tanner graph by progressive edge growth (Hu, Eleftheriou and Arnold, IEEE Trans.
    Inf. Theory 51(1), 2005).  Variables are placed in order of non-decreasing degree;
    the first edge of a variable goes to a check of lowest current degree, every further
    edge to a lowest-degree check among those farthest from the variable in the graph
    built so far: the checks not reached by a breadth-first expansion from the
    variable, taken at the depth where the reached set stops growing, or where it would
    next cover every check.  Ties are broken by a seeded generator.  Returns the
    variables of every check in ascending order."""
    rng = np.random.default_rng(seed)
    order = np.argsort(np.asarray(var_degrees), kind="stable")
    n = len(var_degrees)
    vc = [[] for _ in range(n)]        # checks of each variable
    cv = [[] for _ in range(m)]        # variables of each check
    deg = np.zeros(m, dtype=np.int64)

    def pick(cands: np.ndarray) -> int:
        d = deg[cands]
        best = cands[d == d.min()]
        return int(best[rng.integers(best.size)])

    for v in order:
        for k in range(int(var_degrees[v])):
            if k == 0:
                c = pick(np.arange(m))
            else:
                reached = np.zeros(m, dtype=bool)
                seen_v = {int(v)}
                front = [int(v)]
                while True:
                    new = {c for u in front for c in vc[u] if not reached[c]}
                    if not new:                 # the reached set stopped growing
                        cands = np.nonzero(~reached)[0]
                        break
                    if reached.sum() + len(new) == m:  # the next depth covers all checks
                        cands = np.nonzero(~reached)[0]
                        cands = np.array(sorted(set(cands.tolist()) & new), dtype=np.int64)
                        break
                    reached[list(new)] = True
                    nxt = []
                    for c in new:
                        for u in cv[c]:
                            if u not in seen_v:
                                seen_v.add(u)
                                nxt.append(u)
                    front = nxt
                c = pick(cands)
            vc[v].append(c)
            cv[c].append(int(v))
            deg[c] += 1
    return [sorted(r) for r in cv]


def peg_degrees(n: int, lam: dict[int, float]) -> np.ndarray:
    """Variable degrees for n variables from an edge-perspective distribution
    lambda(x) = sum_i lam[i] x^(i-1): node fractions proportional to lam[i] / i, rounded
    by largest remainder."""
    w = np.array([lam[i] / i for i in sorted(lam)])
    f = w / w.sum() * n
    cnt = np.floor(f).astype(np.int64)
    cnt[np.argsort(-(f - cnt))[: n - cnt.sum()]] += 1
    return np.repeat(np.array(sorted(lam)), cnt)


def code_from_rows(rows: list[list[int]], n: int, name: str = "") -> QCCode:
    """A general sparse code as a QC code with Z = 1 (base entry 0 = a one of H)."""
    base = np.full((len(rows), n), -1, dtype=np.int32)
    for r, vs in enumerate(rows):
        base[r, vs] = 0
    return QCCode(base, 1, name)


def save_rows(path: str, rows: list[list[int]], n: int, comment: str) -> None:
    with open(path, "w") as f:
        f.write(f"# {comment}\n")
        f.write(f"{len(rows)} {n}\n")
        for vs in rows:
            f.write(" ".join(str(v) for v in vs) + "\n")


def load_rows_code(name: str) -> QCCode:
    """A code saved by save_rows (one line of variable indices per check)."""
    with open(os.path.join(CODES_DIR, name + ".txt")) as f:
        lines = [l for l in f if not l.startswith("#")]
    m, n = (int(x) for x in lines[0].split())
    rows = [[int(x) for x in l.split()] for l in lines[1: m + 1]]
    return code_from_rows(rows, n, name)


def code_peg_2048() -> QCCode:
    """Regular (3,6) PEG code, N = 2048, rate 1/2 (seed 5)."""
    return load_rows_code("peg_3_6_n2048_seed5")


def code_peg_irregular_2048() -> QCCode:
    """Irregular PEG code, N = 2048, rate 1/2, lambda(x) = 0.45x + 0.3708x^2 + 0.0307x^3
    + 0.1485x^11 (seed 6)."""
    return load_rows_code("peg_irr_n2048_seed6")


def relift(code: QCCode, Z: int) -> QCCode:
    """Same base graph lifted by a smaller Z (shifts taken mod Z)."""
    b = code.base.copy()
    b[b >= 0] %= Z
    return QCCode(b, Z, name=f"{code.name}_z{Z}")


# ----------------------------------------------------------------------------
# encoders
# ----------------------------------------------------------------------------
def is_lower_triangular(code: QCCode) -> bool:
    """Row r's parity block is column kb + r and every other entry lies left of it."""
    kb = code.nb - code.mb
    if kb < 0:
        return False
    for r in range(code.mb):
        if code.base[r, kb + r] < 0:
            return False
        if (code.base[r, kb + r + 1:] >= 0).any():
            return False
    return True


def encode_lower_triangular(code: QCCode, info: np.ndarray) -> np.ndarray:
    """Systematic encoding by forward substitution over the block rows.

    ``info`` [F, kb*Z] uint8 -> codewords [F, N] uint8.  Requires
    ``is_lower_triangular(code)``; then K = kb*Z and H is full rank.
    """
    if not is_lower_triangular(code):
        raise ValueError("code is not block lower-triangular in its parity part")
    Z, mb, nb = code.Z, code.mb, code.nb
    kb = nb - mb
    info = np.asarray(info, dtype=np.uint8)
    F = info.shape[0]
    x = np.zeros((F, nb, Z), dtype=np.uint8)
    x[:, :kb, :] = info.reshape(F, kb, Z)
    for r in range(mb):
        acc = np.zeros((F, Z), dtype=np.uint8)
        p = kb + r
        for c in range(p):
            s = int(code.base[r, c])
            if s >= 0:
                acc ^= np.roll(x[:, c, :], -s, axis=1)
        x[:, p, :] = np.roll(acc, int(code.base[r, p]), axis=1)
    return x.reshape(F, nb * Z)


def encode_lower_triangular_torch(code: QCCode, info):
    """Torch version of :func:`encode_lower_triangular` (runs on info's device)."""
    import torch

    Z, mb, nb = code.Z, code.mb, code.nb
    kb = nb - mb
    F = info.shape[0]
    x = torch.zeros((F, nb, Z), dtype=torch.uint8, device=info.device)
    x[:, :kb, :] = info.reshape(F, kb, Z)
    for r in range(mb):
        acc = torch.zeros((F, Z), dtype=torch.uint8, device=info.device)
        p = kb + r
        for c in range(p):
            s = int(code.base[r, c])
            if s >= 0:
                acc ^= torch.roll(x[:, c, :], -s, dims=1)
        x[:, p, :] = torch.roll(acc, int(code.base[r, p]), dims=1)
    return x.reshape(F, nb * Z)


def gf2_rank_dense(H: np.ndarray) -> int:
    return gf2_rref(H)[1].size


def gf2_rref(H: np.ndarray):
    """Row-reduce H over GF(2), scanning columns from the right.

    Returns (R, pivot_cols, pivot_rows) with R the reduced matrix.  Scanning
    right-to-left puts pivots in the parity part, so the free (information)
    columns are the leftmost ones whenever the parity part is invertible.
    """
    A = (np.asarray(H, dtype=np.uint8) & 1).copy()
    M, N = A.shape
    piv_cols, piv_rows = [], []
    row = 0
    for c in range(N - 1, -1, -1):
        if row >= M:
            break
        nz = np.nonzero(A[row:, c])[0]
        if nz.size == 0:
            continue
        p = row + int(nz[0])
        if p != row:
            A[[row, p]] = A[[p, row]]
        others = np.nonzero(A[:, c])[0]
        others = others[others != row]
        if others.size:
            A[others] ^= A[row]
        piv_cols.append(c)
        piv_rows.append(row)
        row += 1
    return A, np.array(piv_cols, dtype=np.int64), np.array(piv_rows, dtype=np.int64)


class GF2Encoder:
    """Systematic encoder from Gaussian elimination of a dense H (small codes)."""

    def __init__(self, code: QCCode):
        H = code.dense_H()
        R, pc, pr = gf2_rref(H)
        self.N = code.N
        self.pivot_cols = pc
        free = np.setdiff1d(np.arange(self.N), pc)
        self.info_cols = free
        self.K = free.size
        # pivot variable of row pr[k] = sum over free columns of R[pr[k], free]
        self.A = R[pr][:, free].astype(np.uint8)

    def encode(self, info: np.ndarray) -> np.ndarray:
        info = np.asarray(info, dtype=np.uint8)
        F = info.shape[0]
        x = np.zeros((F, self.N), dtype=np.uint8)
        x[:, self.info_cols] = info
        piv = (info.astype(np.int64) @ self.A.T.astype(np.int64)) & 1
        x[:, self.pivot_cols] = piv.astype(np.uint8)
        return x


# ----------------------------------------------------------------------------
# channel
# ----------------------------------------------------------------------------
def awgn_sigma2(ebn0_db: float, rate: float) -> float:
    """Noise variance per real dimension for BPSK at Eb/N0 (dB) and code rate R."""
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def bpsk_awgn_llr(codewords: np.ndarray, ebn0_db: float, rate: float,
                  rng: np.random.Generator) -> np.ndarray:
    """Channel LLRs 2y/sigma^2 (float32) for BPSK 0->+1, 1->-1 over AWGN."""
    s2 = awgn_sigma2(ebn0_db, rate)
    x = np.asarray(codewords, dtype=np.float64)
    y = (1.0 - 2.0 * x) + np.sqrt(s2) * rng.standard_normal(x.shape)
    return (2.0 * y / s2).astype(np.float32)


@dataclass
class Frames:
    llr: np.ndarray  # float32 [F, N]
    codewords: np.ndarray  # uint8 [F, N]
    ebn0_db: float
    rate: float


def make_frames(code: QCCode, frames: int, ebn0_db: float, seed: int,
                encoder: str = "auto") -> Frames:
    """Host-generated frames: PCG64(seed) draws info bits then the noise.

    ``encoder``: "gf2" (Gaussian elimination), "tri" (block forward
    substitution) or "auto" (gf2 for N <= 4096, tri otherwise).
    """
    rng = np.random.default_rng(seed)
    if encoder == "auto":
        encoder = "gf2" if code.N <= 4096 else "tri"
    if encoder == "gf2":
        enc = GF2Encoder(code)
        K = enc.K
        info = rng.integers(0, 2, size=(frames, K), dtype=np.uint8)
        cw = enc.encode(info)
    elif encoder == "tri":
        K = (code.nb - code.mb) * code.Z
        info = rng.integers(0, 2, size=(frames, K), dtype=np.uint8)
        cw = encode_lower_triangular(code, info)
    elif encoder == "zero":
        K = (code.nb - code.mb) * code.Z
        cw = np.zeros((frames, code.N), dtype=np.uint8)
    else:
        raise ValueError(encoder)
    rate = K / code.N
    llr = bpsk_awgn_llr(cw, ebn0_db, rate, rng)
    return Frames(llr=llr, codewords=cw, ebn0_db=ebn0_db, rate=rate)


def make_frames_torch(code: QCCode, frames: int, ebn0_db, seed: int, device="cuda",
                      zero_codeword: bool = False):
    """Device-generated frames (torch Philox generator), for large batches.

    Random info bits, block forward-substitution encoding, BPSK/AWGN.  ``ebn0_db``
    is a float or a per-frame tensor.  ``zero_codeword`` sends the all-zero codeword
    instead (any code; the decoders are symmetric under codeword sign flips, so error
    statistics do not depend on the codeword).  Returns (llr float32 [F, N], codewords
    uint8).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    K = (code.nb - code.mb) * code.Z
    rate = K / code.N
    if zero_codeword:
        cw = torch.zeros((frames, code.N), device=device, dtype=torch.uint8)
    else:
        if not is_lower_triangular(code):
            raise ValueError("device encoding needs a block lower-triangular code")
        info = torch.randint(0, 2, (frames, K), generator=g, device=device, dtype=torch.uint8)
        cw = encode_lower_triangular_torch(code, info)
    noise = torch.randn((frames, code.N), generator=g, device=device, dtype=torch.float32)
    e = torch.as_tensor(ebn0_db, dtype=torch.float64, device=device)
    s2 = (1.0 / (2.0 * rate * torch.pow(10.0, e / 10.0))).to(torch.float32)
    if s2.ndim == 1:
        s2 = s2[:, None]
    y = (1.0 - 2.0 * cw.to(torch.float32)) + torch.sqrt(s2) * noise
    llr = (2.0 * y / s2).contiguous()
    return llr, cw
