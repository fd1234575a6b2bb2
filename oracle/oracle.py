"""Python view of the plain-C FP64 oracle (``kps_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing in the product
package imports this module, and it imports nothing from the product package.

The oracle follows the paper (Farina & Sandholm, AAAI-22): the payoff matrix
definition of Sec. 2, the river-endgame chance deal and skeleton of Sec. 3 /
Fig. 1, Prop. 1's factors only inside the Technique B identity check of
Sec. 4, and the exploitability measure of Sec. 5.  Vectors are
``[sequence][hand]`` in the oracle's canonical hand order (see
``kps_oracle.h``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kps_oracle.c")
_SRC_TURN = os.path.join(_HERE, "kps_turn_oracle.c")
_LIB = os.path.join(_HERE, "libkps_oracle.so")

MAX_BETS = 8
MAX_BOARD = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC_TURN), os.path.getmtime(os.path.join(_HERE, "kps_oracle.h"))):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                               "-Wall", "-Wno-unused-function", "-o", tmp, _SRC, _SRC_TURN, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Spec(C.Structure):
    _fields_ = [("ranks", C.c_int), ("suits", C.c_int), ("cards_per_hand", C.c_int),
                ("nboard", C.c_int), ("board", C.c_int * MAX_BOARD),
                ("stack", C.c_double * 2), ("contrib0", C.c_double * 2),
                ("nbet", C.c_int), ("bet_frac", C.c_double * MAX_BETS),
                ("raise_cap", C.c_int), ("allow_allin", C.c_int),
                ("mu1", C.POINTER(C.c_double)), ("mu2", C.POINTER(C.c_double)),
                ("strength", C.POINTER(C.c_int)),
                ("use_menu", C.c_int), ("menu_nbet", (C.c_int * 5) * 2),
                ("menu_frac", ((C.c_double * MAX_BETS) * 5) * 2)]


class _TurnSpec(C.Structure):
    _fields_ = [("ranks", C.c_int), ("suits", C.c_int), ("cards_per_hand", C.c_int),
                ("nboard", C.c_int), ("board", C.c_int * MAX_BOARD),
                ("stack", C.c_double * 2), ("contrib0", C.c_double * 2),
                ("nbet_t", C.c_int), ("bet_frac_t", C.c_double * MAX_BETS),
                ("raise_cap_t", C.c_int), ("allow_allin_t", C.c_int),
                ("nbet_r", C.c_int), ("bet_frac_r", C.c_double * MAX_BETS),
                ("raise_cap_r", C.c_int), ("allow_allin_r", C.c_int),
                ("mu1", C.POINTER(C.c_double)), ("mu2", C.POINTER(C.c_double)),
                ("strength", C.POINTER(C.c_int))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.orc_build.restype = P
        L.orc_build.argtypes = [C.POINTER(_Spec)]
        L.orc_free.argtypes = [P]
        L.orc_info.argtypes = [P, P]
        L.orc_beta.restype = C.c_double
        L.orc_regret_floor.argtypes = [P, C.c_int, C.c_double]
        L.orc_regret_floor.restype = C.c_double
        L.orc_rmplus_warm.argtypes = [P, C.c_int, P, P, C.c_double, C.c_int, P, P, P, C.c_int]
        L.orc_rmplus_warm.restype = C.c_double
        L.orc_turn_build.restype = P
        L.orc_turn_build.argtypes = [C.POINTER(_TurnSpec)]
        L.orc_turn_free.argtypes = [P]
        L.orc_turn_info.argtypes = [P, P]
        L.orc_turn_beta.restype = C.c_double
        L.orc_turn_beta.argtypes = [P]
        L.orc_turn_matvec.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int]
        L.orc_turn_entries.argtypes = [P, P, C.c_int, P, P, P, C.c_int, P]
        L.orc_turn_bruteforce.restype = C.c_double
        L.orc_turn_bruteforce.argtypes = [P, P, P]
        L.orc_turn_sequences.argtypes = [P, C.c_int, P, P, P]
        L.orc_turn_seqform.argtypes = [P, C.c_int, P, P]
        L.orc_rmplus_eps.argtypes = [P, C.c_int, C.c_double, P, P]
        L.orc_rmplus_eps.restype = C.c_double
        L.orc_dcfr.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, P, P, P, C.c_int]
        L.orc_dcfr.restype = C.c_double
        L.orc_beta.argtypes = [P]
        L.orc_pot0.restype = C.c_double
        L.orc_pot0.argtypes = [P]
        L.orc_hands.argtypes = [P, P]
        L.orc_terminals.argtypes = [P] + [P] * 6
        L.orc_sequences.argtypes = [P, C.c_int, P, P, P, P, P]
        L.orc_find_terminal.restype = C.c_int
        L.orc_find_terminal.argtypes = [P, C.c_char_p]
        L.orc_dense_A.argtypes = [P, P]
        for f in (L.orc_matvec_A, L.orc_matvec_AT):
            f.argtypes = [P, P, P, C.c_int, C.c_int]
        for f in (L.orc_matvec_A_entries, L.orc_matvec_AT_entries):
            f.argtypes = [P, P, C.c_int, P, P, P, P]
        L.orc_bruteforce_value.restype = C.c_double
        L.orc_bruteforce_value.argtypes = [P, P, P]
        L.orc_seqform.argtypes = [P, C.c_int, P, P]
        L.orc_technique_b.restype = C.c_double
        L.orc_technique_b.argtypes = [P, P]
        L.orc_technique_b_counts.argtypes = [P, P]
        L.orc_rmplus.restype = C.c_double
        L.orc_rmplus.argtypes = [P, C.c_int, P, P, P, P, P, C.c_int]
        L.orc_exploitability.restype = C.c_double
        L.orc_exploitability.argtypes = [P, P, P, P, P]
        L.orc_value.restype = C.c_double
        L.orc_value.argtypes = [P, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleGame:
    """One river endgame, built by the oracle from a plain spec dict.

    spec keys: ranks, suits, cards_per_hand, board (list of card ids),
    stack (2), contrib0 (2), bet_frac (list), raise_cap (int, <0 none),
    allow_allin (bool), strength (per canonical hand), mu1/mu2 (optional),
    menu (optional: menu[player][situation] = list of fractions, situations
    first action / after a check / facing the first bet / facing one raise /
    facing two or more raises).
    """

    def __init__(self, spec: dict):
        L = lib()
        s = _Spec()
        s.ranks, s.suits = int(spec["ranks"]), int(spec["suits"])
        s.cards_per_hand = int(spec["cards_per_hand"])
        board = list(spec.get("board", []))
        s.nboard = len(board)
        for i, c in enumerate(board):
            s.board[i] = int(c)
        s.stack[0], s.stack[1] = [float(v) for v in spec["stack"]]
        s.contrib0[0], s.contrib0[1] = [float(v) for v in spec["contrib0"]]
        fr = list(spec.get("bet_frac", []))
        s.nbet = len(fr)
        for i, f in enumerate(fr):
            s.bet_frac[i] = float(f)
        s.raise_cap = int(spec.get("raise_cap", -1))
        s.allow_allin = 1 if spec.get("allow_allin", False) else 0
        if spec.get("menu") is not None:
            s.use_menu = 1
            for p in range(2):
                for k in range(5):
                    fr = list(spec["menu"][p][k])
                    s.menu_nbet[p][k] = len(fr)
                    for i, f in enumerate(fr):
                        s.menu_frac[p][k][i] = float(f)
        self._strength = np.ascontiguousarray(spec["strength"], dtype=np.int32)
        self._mu1 = None if spec.get("mu1") is None else np.ascontiguousarray(spec["mu1"], dtype=np.float64)
        self._mu2 = None if spec.get("mu2") is None else np.ascontiguousarray(spec["mu2"], dtype=np.float64)
        s.strength = self._strength.ctypes.data_as(C.POINTER(C.c_int))
        s.mu1 = self._mu1.ctypes.data_as(C.POINTER(C.c_double)) if self._mu1 is not None else None
        s.mu2 = self._mu2.ctypes.data_as(C.POINTER(C.c_double)) if self._mu2 is not None else None
        self._g = L.orc_build(C.byref(s))
        if not self._g:
            raise ValueError("oracle rejected the game spec")
        info = np.zeros(10, dtype=np.int32)
        L.orc_info(self._g, _p(info))
        (self.H, self.n1, self.n2, self.T, self.TF, self.TS, self.nnodes,
         self.ncards_left, self.np1, self.np2) = [int(v) for v in info]
        self.k = int(spec["cards_per_hand"])
        self.beta = L.orc_beta(self._g)
        self.pot0 = L.orc_pot0(self._g)

    def __del__(self):
        if getattr(self, "_g", None):
            lib().orc_free(self._g)
            self._g = None

    # ---------------------------------------------------------- structure
    def hands(self) -> np.ndarray:
        out = np.zeros(self.H * self.k, dtype=np.int32)
        lib().orc_hands(self._g, _p(out))
        return out.reshape(self.H, self.k)

    def terminals(self) -> dict:
        T = self.T
        s1, s2, kind, folder = (np.zeros(T, np.int32) for _ in range(4))
        c1, c2 = np.zeros(T), np.zeros(T)
        lib().orc_terminals(self._g, _p(s1), _p(s2), _p(kind), _p(folder), _p(c1), _p(c2))
        return dict(s1=s1, s2=s2, kind=kind, folder=folder, c1=c1, c2=c2)

    def sequences(self, p: int) -> dict:
        n = self.n1 if p == 0 else self.n2
        npn = self.np1 if p == 0 else self.np2
        node, parent, action = (np.zeros(n, np.int32) for _ in range(3))
        amount = np.zeros(n)
        nact = np.zeros(npn, np.int32)
        lib().orc_sequences(self._g, p, _p(node), _p(parent), _p(action), _p(amount), _p(nact))
        return dict(node=node, parent=parent, action=action, amount=amount, nact=nact)

    def find_terminal(self, path: str) -> int:
        return lib().orc_find_terminal(self._g, path.encode())

    # ------------------------------------------------------------ algebra
    def dense_A(self) -> np.ndarray:
        A = np.zeros((self.H * self.n1, self.H * self.n2))
        lib().orc_dense_A(self._g, _p(A))
        return A

    def matvec_A(self, y: np.ndarray, nthreads: int = 0) -> np.ndarray:
        y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, self.n2, self.H)
        out = np.zeros((y.shape[0], self.n1, self.H))
        lib().orc_matvec_A(self._g, _p(y), _p(out), y.shape[0], nthreads)
        return out

    def matvec_AT(self, x: np.ndarray, nthreads: int = 0) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, self.n1, self.H)
        out = np.zeros((x.shape[0], self.n2, self.H))
        lib().orc_matvec_AT(self._g, _p(x), _p(out), x.shape[0], nthreads)
        return out

    def matvec_entries(self, v: np.ndarray, b, s, h, transpose: bool = False) -> np.ndarray:
        nin = self.n1 if transpose else self.n2
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, nin, self.H)
        b, s, h = (np.ascontiguousarray(a, dtype=np.int32) for a in (b, s, h))
        out = np.zeros(len(b))
        f = lib().orc_matvec_AT_entries if transpose else lib().orc_matvec_A_entries
        f(self._g, _p(v), len(b), _p(b), _p(s), _p(h), _p(out))
        return out

    def bruteforce_value(self, beh1: np.ndarray, beh2: np.ndarray) -> float:
        b1 = np.ascontiguousarray(beh1, dtype=np.float64)
        b2 = np.ascontiguousarray(beh2, dtype=np.float64)
        return lib().orc_bruteforce_value(self._g, _p(b1), _p(b2))

    def seqform(self, p: int, beh: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(beh, dtype=np.float64)
        x = np.zeros_like(b)
        lib().orc_seqform(self._g, p, _p(b), _p(x))
        return x

    def technique_b(self):
        cnt = np.zeros(9, dtype=np.int64)
        err = lib().orc_technique_b(self._g, _p(cnt))
        return err, cnt

    def technique_b_counts(self) -> np.ndarray:
        cnt = np.zeros(9, dtype=np.int64)
        lib().orc_technique_b_counts(self._g, _p(cnt))
        return cnt

    def regret_floor(self, p: int, eps: float) -> float:
        """eps * V_p, V_p the bound on player p's counterfactual values."""
        return lib().orc_regret_floor(self._g, p, eps)

    def rmplus(self, iters: int, beh1=None, beh2=None, trace_every: int = 0):
        avg1 = np.zeros((self.n1, self.H))
        avg2 = np.zeros((self.n2, self.H))
        trace = np.zeros(max(iters, 1))
        b1 = None if beh1 is None else np.ascontiguousarray(beh1, dtype=np.float64)
        b2 = None if beh2 is None else np.ascontiguousarray(beh2, dtype=np.float64)
        e = lib().orc_rmplus(self._g, iters, _p(b1), _p(b2), _p(avg1), _p(avg2), _p(trace), trace_every)
        return e, avg1, avg2, trace[:iters]

    def rmplus_warm(self, iters: int, beh1, beh2, kappa: float, t0: int, trace_every: int = 0):
        """RM+ started warm (see orc_rmplus_warm)."""
        avg1 = np.zeros((self.n1, self.H))
        avg2 = np.zeros((self.n2, self.H))
        trace = np.zeros(max(iters, 1))
        b1 = None if beh1 is None else np.ascontiguousarray(beh1, dtype=np.float64)
        b2 = None if beh2 is None else np.ascontiguousarray(beh2, dtype=np.float64)
        e = lib().orc_rmplus_warm(self._g, iters, _p(b1), _p(b2), kappa, t0, _p(avg1), _p(avg2), _p(trace),
                                  trace_every)
        return e, avg1, avg2, trace[:iters]

    def rmplus_eps(self, iters: int, eps: float):
        """RM+ from uniform strategies with the regret-matching noise floor
        eps * V_p (eps = 0: textbook RM+); returns (expl, avg1, avg2)."""
        avg1 = np.zeros((self.n1, self.H))
        avg2 = np.zeros((self.n2, self.H))
        e = lib().orc_rmplus_eps(self._g, iters, float(eps), _p(avg1), _p(avg2))
        return e, avg1, avg2

    def dcfr(self, iters: int, alpha: float = 1.5, beta: float = 0.0, gamma: float = 2.0, trace_every: int = 0):
        """Discounted CFR from uniform strategies (see orc_dcfr)."""
        avg1 = np.zeros((self.n1, self.H))
        avg2 = np.zeros((self.n2, self.H))
        trace = np.zeros(max(iters, 1))
        e = lib().orc_dcfr(self._g, iters, alpha, beta, gamma, _p(avg1), _p(avg2), _p(trace), trace_every)
        return e, avg1, avg2, trace[:iters]

    def exploitability(self, x: np.ndarray, y: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        b1, b2 = C.c_double(), C.c_double()
        e = lib().orc_exploitability(self._g, _p(x), _p(y), C.byref(b1), C.byref(b2))
        return e, b1.value, b2.value

    def value(self, x: np.ndarray, y: np.ndarray) -> float:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        return lib().orc_value(self._g, _p(x), _p(y))


class OracleTurn:
    """A turn endgame (turn round, river card, river round) built by the
    oracle from a spec dict: ranks, suits, cards_per_hand, board (the turn
    board), stack, contrib0, bet_frac_t / raise_cap_t / allow_allin_t (turn
    round), bet_frac_r / raise_cap_r / allow_allin_r (river round), mu1 /
    mu2 (per hand, optional) and strength [ranks*suits][H] (hand strength
    with each river card).  Vectors are [sequence][hand] in the layout of
    kps_oracle.h (turn sequences, then the (ending, river card) blocks)."""

    def __init__(self, spec: dict):
        L = lib()
        s = _TurnSpec()
        s.ranks, s.suits = int(spec["ranks"]), int(spec["suits"])
        s.cards_per_hand = int(spec["cards_per_hand"])
        board = list(spec["board"])
        s.nboard = len(board)
        for i, c in enumerate(board):
            s.board[i] = int(c)
        s.stack[0], s.stack[1] = [float(v) for v in spec["stack"]]
        s.contrib0[0], s.contrib0[1] = [float(v) for v in spec["contrib0"]]
        for tag in ("t", "r"):
            fr = list(spec["bet_frac_" + tag])
            setattr(s, "nbet_" + tag, len(fr))
            arr = getattr(s, "bet_frac_" + tag)
            for i, f in enumerate(fr):
                arr[i] = float(f)
            setattr(s, "raise_cap_" + tag, int(spec["raise_cap_" + tag]))
            setattr(s, "allow_allin_" + tag, 1 if spec.get("allow_allin_" + tag, False) else 0)
        self._strength = np.ascontiguousarray(spec["strength"], dtype=np.int32)
        self._mu1 = None if spec.get("mu1") is None else np.ascontiguousarray(spec["mu1"], dtype=np.float64)
        self._mu2 = None if spec.get("mu2") is None else np.ascontiguousarray(spec["mu2"], dtype=np.float64)
        s.strength = self._strength.ctypes.data_as(C.POINTER(C.c_int))
        s.mu1 = self._mu1.ctypes.data_as(C.POINTER(C.c_double)) if self._mu1 is not None else None
        s.mu2 = self._mu2.ctypes.data_as(C.POINTER(C.c_double)) if self._mu2 is not None else None
        self._g = L.orc_turn_build(C.byref(s))
        if not self._g:
            raise ValueError("oracle rejected the turn spec")
        info = np.zeros(9, dtype=np.int32)
        L.orc_turn_info(self._g, _p(info))
        (self.H, self.n1, self.n2, self.T, self.endings, self.blocks, self.nturn1, self.nturn2,
         self.N) = [int(v) for v in info]
        self.beta = L.orc_turn_beta(self._g)

    def __del__(self):
        if getattr(self, "_g", None):
            lib().orc_turn_free(self._g)
            self._g = None

    def sequences(self, p: int) -> dict:
        n = self.n1 if p == 0 else self.n2
        parent, node, nact = (np.zeros(n, np.int32) for _ in range(3))
        lib().orc_turn_sequences(self._g, p, _p(parent), _p(node), _p(nact))
        return dict(parent=parent, node=node, nact=nact)

    def matvec(self, v: np.ndarray, transpose: bool = False, nthreads: int = 0) -> np.ndarray:
        nin, nout = (self.n1, self.n2) if transpose else (self.n2, self.n1)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, nin, self.H)
        out = np.zeros((v.shape[0], nout, self.H))
        lib().orc_turn_matvec(self._g, _p(v), _p(out), v.shape[0], 1 if transpose else 0, nthreads)
        return out

    def entries(self, v: np.ndarray, b, s, h, transpose: bool = False) -> np.ndarray:
        nin = self.n1 if transpose else self.n2
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, nin, self.H)
        b, s, h = (np.ascontiguousarray(a, dtype=np.int32) for a in (b, s, h))
        out = np.zeros(len(b))
        lib().orc_turn_entries(self._g, _p(v), len(b), _p(b), _p(s), _p(h), 1 if transpose else 0, _p(out))
        return out

    def bruteforce_value(self, beh1: np.ndarray, beh2: np.ndarray) -> float:
        b1 = np.ascontiguousarray(beh1, dtype=np.float64)
        b2 = np.ascontiguousarray(beh2, dtype=np.float64)
        return lib().orc_turn_bruteforce(self._g, _p(b1), _p(b2))

    def seqform(self, p: int, beh: np.ndarray) -> np.ndarray:
        b = np.ascontiguousarray(beh, dtype=np.float64)
        x = np.zeros_like(b)
        lib().orc_turn_seqform(self._g, p, _p(b), _p(x))
        return x

