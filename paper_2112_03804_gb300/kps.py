"""Python binding of the C ABI in ``include/kps.h`` (argument marshalling only).

Every computation runs in ``libkps.so``; this module converts Python values
to the C structs and pointers the ABI takes.  Vector arguments may be torch
tensors (their ``data_ptr()`` is passed) or raw integer addresses.  The
library must have been built (``paper_2112_03804_gb300.build.build()``);
importing the binding without it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkps.so")

MAX_BETS = 8
MAX_BOARD = 8

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP, ENUMERIC = range(7)
F32, F64, BF16, F16 = 0, 1, 2, 3
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTSUP", 6: "ENUMERIC"}


class KpsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


SITUATIONS = 5


class BetMenu(C.Structure):
    """kps_bet_menu: per player and situation (first action, after a check,
    facing the first bet, facing one raise, facing two or more raises) the
    bet/raise pot fractions."""
    _fields_ = [("nbet", (C.c_int32 * SITUATIONS) * 2),
                ("bet_frac", ((C.c_double * MAX_BETS) * SITUATIONS) * 2)]


class GameSpec(C.Structure):
    _fields_ = [("ranks", C.c_int32), ("suits", C.c_int32), ("cards_per_hand", C.c_int32),
                ("nboard", C.c_int32), ("board", C.c_int32 * MAX_BOARD),
                ("stack", C.c_double * 2), ("contrib0", C.c_double * 2),
                ("nbet", C.c_int32), ("bet_frac", C.c_double * MAX_BETS),
                ("raise_cap", C.c_int32), ("allow_allin", C.c_int32),
                ("mu1", C.POINTER(C.c_double)), ("mu2", C.POINTER(C.c_double)),
                ("strength", C.POINTER(C.c_int32)), ("menu", C.POINTER(BetMenu))]


class TurnSpec(C.Structure):
    _fields_ = [("ranks", C.c_int32), ("suits", C.c_int32), ("cards_per_hand", C.c_int32),
                ("nboard", C.c_int32), ("board", C.c_int32 * MAX_BOARD),
                ("stack", C.c_double * 2), ("contrib0", C.c_double * 2),
                ("nbet_turn", C.c_int32), ("bet_frac_turn", C.c_double * MAX_BETS),
                ("raise_cap_turn", C.c_int32), ("allow_allin_turn", C.c_int32),
                ("nbet_river", C.c_int32), ("bet_frac_river", C.c_double * MAX_BETS),
                ("raise_cap_river", C.c_int32), ("allow_allin_river", C.c_int32),
                ("mu1", C.POINTER(C.c_double)), ("mu2", C.POINTER(C.c_double)),
                ("strength", C.POINTER(C.c_int32))]


class Info(C.Structure):
    _fields_ = [("H", C.c_int32), ("hs", C.c_int32), ("n1", C.c_int32), ("n2", C.c_int32),
                ("T", C.c_int32), ("T_fold", C.c_int32), ("T_showdown", C.c_int32),
                ("ncards", C.c_int32), ("cards_per_hand", C.c_int32),
                ("nodes1", C.c_int32), ("nodes2", C.c_int32), ("max_tie", C.c_int32),
                ("beta", C.c_double), ("pot0", C.c_double),
                ("nnz_A", C.c_int64), ("nnz_Ahat", C.c_int64), ("nnz_U", C.c_int64),
                ("nnz_M", C.c_int64), ("nnz_V", C.c_int64), ("pp_nnz_Ahat", C.c_int64),
                ("pp_nnz_U", C.c_int64), ("pp_nnz_M", C.c_int64), ("pp_nnz_V", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchShape(C.Structure):
    _fields_ = [("warps", C.c_int32), ("grid", C.c_int32), ("schedule", C.c_int32), ("kernel", C.c_int32),
                ("ms_per_pair", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTED = ["kps_sparsify", "kps_game_destroy", "kps_game_info", "kps_game_hands",
            "kps_game_sequences", "kps_game_terminals", "kps_game_upload", "kps_game_kernel",
            "kps_matvec_A", "kps_matvec_AT", "kps_matvec_A_host", "kps_matvec_AT_host",
            "kps_matvec_A_static_scratch",
            "kps_batch_create", "kps_batch_destroy", "kps_batch_offsets", "kps_batch_matvec_A",
            "kps_batch_matvec_AT", "kps_batch_tune", "kps_batch_shape_get", "kps_batch_shape_set", "kps_partition",
            "kps_solver_create", "kps_solver_destroy", "kps_solver_reset", "kps_solver_warm_start",
            "kps_solver_set_method", "kps_solver_step", "kps_solver_status", "kps_solver_state_bytes",
            "kps_solver_save", "kps_solver_load",
            "kps_solver_iterations", "kps_solver_average", "kps_solver_strategy", "kps_solver_exploitability",
            "kps_solver_exploitability_estimate",
            "kps_warm_num_queries", "kps_warm_features", "kps_warm_targets", "kps_warm_scatter",
            "kps_warm_predict",
            "kps_mlp_create", "kps_mlp_destroy", "kps_mlp_num_params", "kps_mlp_get", "kps_mlp_set",
            "kps_mlp_forward", "kps_mlp_gradients", "kps_mlp_adam", "kps_mlp_state_bytes", "kps_mlp_save",
            "kps_mlp_load",
            "kps_turn_create", "kps_turn_destroy", "kps_turn_info", "kps_turn_offsets", "kps_turn_block",
            "kps_turn_matvec_A", "kps_turn_matvec_AT", "kps_turn_batch", "kps_device_status",
            "kps_tb_create", "kps_tb_destroy", "kps_tb_sizes", "kps_tb_export", "kps_tb_matvec",
            "kps_last_error", "kps_version"]

_lib = None


def lib():
    """Load libkps.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2112_03804_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.kps_sparsify.argtypes = [C.POINTER(GameSpec), C.POINTER(C.c_void_p)]
        L.kps_game_destroy.argtypes = [P]
        L.kps_game_info.argtypes = [P, C.POINTER(Info)]
        L.kps_game_hands.argtypes = [P, P, P]
        L.kps_game_sequences.argtypes = [P, C.c_int32, P, P, P, P, P]
        L.kps_game_terminals.argtypes = [P, P, P, P, P, P, P]
        L.kps_game_upload.argtypes = [P, P]
        L.kps_game_kernel.argtypes = [P, C.c_int32, C.POINTER(C.c_int32)]
        for f in (L.kps_matvec_A, L.kps_matvec_AT, L.kps_matvec_A_host, L.kps_matvec_AT_host,
                  L.kps_matvec_A_static_scratch):
            f.argtypes = [P, P, P, C.c_int32, C.c_int, P]
        L.kps_batch_create.argtypes = [P, C.c_int32, C.POINTER(C.c_void_p)]
        L.kps_batch_destroy.argtypes = [P]
        L.kps_batch_offsets.argtypes = [P, C.c_int32, P]
        L.kps_batch_matvec_A.argtypes = [P, P, P, C.c_int, P]
        L.kps_batch_matvec_AT.argtypes = [P, P, P, C.c_int, P]
        L.kps_batch_tune.argtypes = [P, C.c_int, P, C.POINTER(BatchShape)]
        L.kps_batch_shape_get.argtypes = [P, C.c_int, C.POINTER(BatchShape)]
        L.kps_batch_shape_set.argtypes = [P, C.c_int, C.POINTER(BatchShape)]
        L.kps_partition.argtypes = [P, C.c_int32, C.c_int32, P]
        L.kps_solver_create.argtypes = [P, C.c_int, C.POINTER(C.c_void_p)]
        L.kps_solver_destroy.argtypes = [P]
        L.kps_solver_reset.argtypes = [P, P, P, P]
        L.kps_solver_step.argtypes = [P, C.c_int32, P]
        L.kps_solver_status.argtypes = [P]
        L.kps_turn_create.argtypes = [C.POINTER(TurnSpec), C.POINTER(C.c_void_p)]
        L.kps_turn_destroy.argtypes = [P]
        L.kps_turn_info.argtypes = [P, P]
        L.kps_turn_offsets.argtypes = [P, C.c_int32, P]
        L.kps_turn_block.argtypes = [P, C.c_int32, P, P, P]
        L.kps_turn_matvec_A.argtypes = [P, P, P, C.c_int, P]
        L.kps_turn_matvec_AT.argtypes = [P, P, P, C.c_int, P]
        L.kps_turn_batch.argtypes = [P, C.POINTER(C.c_void_p)]
        L.kps_device_status.argtypes = [P]
        L.kps_solver_state_bytes.argtypes = [P, C.POINTER(C.c_int64)]
        L.kps_solver_save.argtypes = [P, P, C.c_int64, P]
        L.kps_solver_load.argtypes = [P, P, C.c_int64, P]
        L.kps_mlp_state_bytes.argtypes = [P, C.POINTER(C.c_int64)]
        L.kps_mlp_save.argtypes = [P, P, C.c_int64]
        L.kps_mlp_load.argtypes = [P, P, C.c_int64]
        L.kps_solver_iterations.argtypes = [P, C.POINTER(C.c_int64)]
        L.kps_solver_average.argtypes = [P, C.c_int32, P, P, P]
        L.kps_solver_exploitability.argtypes = [P, P, P, P, P]
        L.kps_solver_strategy.argtypes = [P, P, P, P]
        L.kps_solver_exploitability_estimate.argtypes = [P, P, P]
        L.kps_solver_warm_start.argtypes = [P, P, P, C.c_double, C.c_int32, P]
        L.kps_solver_set_method.argtypes = [P, C.c_int32, C.c_double, C.c_double, C.c_double]
        L.kps_warm_num_queries.argtypes = [P, C.POINTER(C.c_int64)]
        L.kps_warm_features.argtypes = [P, P, C.c_int64, C.c_int32, P, P, P]
        L.kps_warm_targets.argtypes = [P, P, P, P, P, P, C.c_int64, C.c_int32, P, P, P]
        L.kps_warm_scatter.argtypes = [P, P, P, C.c_int64, C.c_int32, P, P, P]
        L.kps_warm_predict.argtypes = [P, P, P, P, P]
        L.kps_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]
        L.kps_mlp_destroy.argtypes = [P]
        L.kps_mlp_num_params.argtypes = [P, C.POINTER(C.c_int64)]
        L.kps_mlp_get.argtypes = [P, C.c_int32, P]
        L.kps_mlp_set.argtypes = [P, P]
        L.kps_mlp_forward.argtypes = [P, P, C.c_int32, P, P, P]
        L.kps_mlp_gradients.argtypes = [P, P, C.c_int32, P, P, P, C.c_float, P, P]
        L.kps_mlp_adam.argtypes = [P, C.c_float, C.c_float, C.c_float, C.c_float, P]
        L.kps_tb_create.argtypes = [P, C.POINTER(C.c_void_p)]
        L.kps_tb_destroy.argtypes = [P]
        L.kps_tb_sizes.argtypes = [P, P]
        L.kps_tb_export.argtypes = [P, C.c_int, P, P, P, P]
        L.kps_tb_matvec.argtypes = [P, P, P, C.c_int32, C.c_int, C.c_int32, P]
        for name in EXPORTED:
            if name not in ("kps_last_error", "kps_version"):
                getattr(L, name).restype = C.c_int
        L.kps_last_error.restype = C.c_char_p
        L.kps_version.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise KpsError(status, lib().kps_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


_TORCH_DT = {}


def _dtype_code(t, dtype):
    if dtype is not None:
        return dtype
    import torch
    m = {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16, torch.float16: F16}
    return m[t.dtype]


class Game:
    """A river endgame built by ``kps_sparsify`` (see ``include/kps.h``)."""

    def __init__(self, spec: dict):
        s = GameSpec()
        s.ranks, s.suits = int(spec["ranks"]), int(spec["suits"])
        s.cards_per_hand = int(spec["cards_per_hand"])
        board = list(spec.get("board", []))
        if len(board) > MAX_BOARD:
            raise ValueError("board too long")
        s.nboard = len(board)
        for i, c in enumerate(board):
            s.board[i] = int(c)
        s.stack[0], s.stack[1] = [float(v) for v in spec["stack"]]
        s.contrib0[0], s.contrib0[1] = [float(v) for v in spec["contrib0"]]
        fr = list(spec.get("bet_frac", []))
        if len(fr) > MAX_BETS:
            raise ValueError("too many bet sizes")
        s.nbet = len(fr)
        for i, f in enumerate(fr):
            s.bet_frac[i] = float(f)
        s.raise_cap = int(spec.get("raise_cap", -1))
        s.allow_allin = 1 if spec.get("allow_allin", False) else 0
        # optional menu: spec["menu"][player][situation] = list of fractions
        self._menu = None
        if spec.get("menu") is not None:
            m = BetMenu()
            for p in range(2):
                for k in range(SITUATIONS):
                    fr = list(spec["menu"][p][k])
                    if len(fr) > MAX_BETS:
                        raise ValueError("too many bet sizes in the menu")
                    m.nbet[p][k] = len(fr)
                    for i, f in enumerate(fr):
                        m.bet_frac[p][k][i] = float(f)
            self._menu = m
            s.menu = C.pointer(m)
        self._strength = np.ascontiguousarray(spec["strength"], dtype=np.int32)
        mu1, mu2 = spec.get("mu1"), spec.get("mu2")
        self._mu1 = None if mu1 is None else np.ascontiguousarray(mu1, dtype=np.float64)
        self._mu2 = None if mu2 is None else np.ascontiguousarray(mu2, dtype=np.float64)
        s.strength = self._strength.ctypes.data_as(C.POINTER(C.c_int32))
        s.mu1 = self._mu1.ctypes.data_as(C.POINTER(C.c_double)) if self._mu1 is not None else None
        s.mu2 = self._mu2.ctypes.data_as(C.POINTER(C.c_double)) if self._mu2 is not None else None
        h = C.c_void_p()
        _check(lib().kps_sparsify(C.byref(s), C.byref(h)))
        self._h = h
        self._info = None

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kps_game_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        if self._info is None:
            i = Info()
            _check(lib().kps_game_info(self._h, C.byref(i)))
            self._info = i.as_dict()
        return self._info

    def hands(self):
        inf = self.info()
        cards = np.zeros(inf["H"] * inf["cards_per_hand"], dtype=np.int32)
        canon = np.zeros(inf["H"], dtype=np.int32)
        _check(lib().kps_game_hands(self._h, cards.ctypes.data, canon.ctypes.data))
        return cards.reshape(inf["H"], inf["cards_per_hand"]), canon

    def sequences(self, player: int) -> dict:
        inf = self.info()
        n = inf["n1"] if player == 0 else inf["n2"]
        nn = inf["nodes1"] if player == 0 else inf["nodes2"]
        node, parent, action = (np.zeros(n, np.int32) for _ in range(3))
        amount = np.zeros(n)
        nact = np.zeros(nn, np.int32)
        _check(lib().kps_game_sequences(self._h, player, node.ctypes.data, parent.ctypes.data,
                                        action.ctypes.data, amount.ctypes.data, nact.ctypes.data))
        return dict(node=node, parent=parent, action=action, amount=amount, nact=nact)

    def terminals(self) -> dict:
        T = self.info()["T"]
        s1, s2, kind, folder = (np.zeros(T, np.int32) for _ in range(4))
        c1, c2 = np.zeros(T), np.zeros(T)
        _check(lib().kps_game_terminals(self._h, s1.ctypes.data, s2.ctypes.data, kind.ctypes.data,
                                        folder.ctypes.data, c1.ctypes.data, c2.ctypes.data))
        return dict(s1=s1, s2=s2, kind=kind, folder=folder, c1=c1, c2=c2)

    def upload(self, stream=None):
        _check(lib().kps_game_upload(self._h, _stream(stream)))

    def kernel(self, direction: int) -> str:
        """kps_game_kernel: name of the kernel that ran the last product of
        a direction (0 = A*y, 1 = A^T*x); "" before the first."""
        k = C.c_int32(0)
        _check(lib().kps_game_kernel(self._h, int(direction), C.byref(k)))
        return KERNEL_NAMES.get(k.value, "")


def sparsify(spec: dict) -> Game:
    return Game(spec)


def matvec_A(game: Game, y, out, batch: int, dtype=None, stream=None):
    """out[b] = A y[b]; y [batch][n2][hs], out [batch][n1][hs] on the device."""
    _check(lib().kps_matvec_A(game._h, _ptr(y), _ptr(out), int(batch), _dtype_code(y, dtype), _stream(stream)))


def matvec_AT(game: Game, x, out, batch: int, dtype=None, stream=None):
    """out[b] = A^T x[b]; x [batch][n1][hs], out [batch][n2][hs] on the device."""
    _check(lib().kps_matvec_AT(game._h, _ptr(x), _ptr(out), int(batch), _dtype_code(x, dtype), _stream(stream)))


def matvec_A_host(game: Game, y, out, batch: int, dtype: int, stream=None):
    """Same as matvec_A with host buffers (copies inside, synchronous)."""
    _check(lib().kps_matvec_A_host(game._h, _ptr(y), _ptr(out), int(batch), dtype, _stream(stream)))


def matvec_AT_host(game: Game, x, out, batch: int, dtype: int, stream=None):
    _check(lib().kps_matvec_AT_host(game._h, _ptr(x), _ptr(out), int(batch), dtype, _stream(stream)))


class TechniqueB:
    """Technique B's explicit factors of a game's A (Sec. 4), built on the
    host: A = Ahat + U M^-1 V^T.  `sizes()` gives R, C, m and the nonzero
    counts; `export(which)` a factor as (shape, rowptr, col, val) numpy
    arrays (0 Ahat, 1 U, 2 M, 3 V^T); `matvec` the GPU product with this
    library's kernels (backend 0) or cuSPARSE (backend 1)."""

    AHAT, U, M, VT = 0, 1, 2, 3

    def __init__(self, game: Game):
        self._game = game           # the factors refer to the game's tables
        h = C.c_void_p()
        _check(lib().kps_tb_create(game._h, C.byref(h)))
        self._h = h.value

    def sizes(self) -> dict:
        a = np.zeros(7, dtype=np.int64)
        _check(lib().kps_tb_sizes(self._h, _ptr(a)))
        return dict(zip(("R", "C", "m", "nnz_Ahat", "nnz_U", "nnz_M", "nnz_V"), (int(x) for x in a)))

    def export(self, which: int):
        shape = np.zeros(3, dtype=np.int64)
        _check(lib().kps_tb_export(self._h, which, _ptr(shape), None, None, None))
        rows, cols, nnz = (int(x) for x in shape)
        rowptr = np.zeros(rows + 1, dtype=np.int32)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1), dtype=np.float64)
        _check(lib().kps_tb_export(self._h, which, None, _ptr(rowptr), _ptr(col), _ptr(val)))
        return (rows, cols), rowptr, col[:nnz], val[:nnz]

    def matvec(self, y, out, batch: int, backend: int = 0, dtype=None, stream=None):
        """out[b] = (Ahat + U M^-1 V^T) y[b]; y [batch][n2][hs], out [batch][n1][hs] on the device."""
        _check(lib().kps_tb_matvec(self._h, _ptr(y), _ptr(out), int(batch), _dtype_code(y, dtype), int(backend),
                                   _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().kps_tb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STATIC_SCRATCH_FLOATS = 4194304
BATCH_TMEM, BATCH_STAGED = 0, 1
KERNEL_NAMES = {1: "tma", 2: "tmem", 3: "vec", 4: "fast", 5: "general"}


def matvec_A_static_scratch(game: Game, y, out, batch: int, dtype=None, stream=None):
    """kps_matvec_A_static_scratch: BF16/FP16 A*y with no device allocation
    (statically reserved scratch; see include/kps.h for the contract)."""
    _check(lib().kps_matvec_A_static_scratch(game._h, _ptr(y), _ptr(out), int(batch), _dtype_code(y, dtype),
                                             _stream(stream)))


class Batch:
    """Several games whose products run as one persistent launch
    (``kps_batch_*``).  Keeps the games alive while it lives."""

    def __init__(self, games):
        self.games = list(games)
        arr = (C.c_void_p * len(self.games))(*[g.handle for g in self.games])
        h = C.c_void_p()
        _check(lib().kps_batch_create(arr, len(self.games), C.byref(h)))
        self._h = h

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kps_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def offsets(self, player: int) -> np.ndarray:
        off = np.zeros(len(self.games) + 1, dtype=np.int64)
        _check(lib().kps_batch_offsets(self._h, player, off.ctypes.data))
        return off

    def matvec_A(self, y, out, dtype=None, stream=None):
        _check(lib().kps_batch_matvec_A(self._h, _ptr(y), _ptr(out), _dtype_code(y, dtype), _stream(stream)))

    def matvec_AT(self, x, out, dtype=None, stream=None):
        _check(lib().kps_batch_matvec_AT(self._h, _ptr(x), _ptr(out), _dtype_code(x, dtype), _stream(stream)))

    def tune(self, dtype: int, stream=None) -> dict:
        sh = BatchShape()
        _check(lib().kps_batch_tune(self._h, dtype, _stream(stream), C.byref(sh)))
        return sh.as_dict()

    def shape(self, dtype: int) -> dict:
        sh = BatchShape()
        _check(lib().kps_batch_shape_get(self._h, dtype, C.byref(sh)))
        return sh.as_dict()

    def set_shape(self, dtype: int, warps: int, grid: int, schedule: int, kernel: int = 0):
        """kernel: BATCH_TMEM (0) or BATCH_STAGED (1, FP32, 4 warps)."""
        sh = BatchShape(warps, grid, schedule, kernel, 0.0)
        _check(lib().kps_batch_shape_set(self._h, dtype, C.byref(sh)))


def device_status(stream=None):
    """Synchronises `stream`; raises KpsError(ETIMEOUT) when a bounded
    device wait gave up since the last call (``kps_device_status``)."""
    _check(lib().kps_device_status(_stream(stream)))


def partition(weights, parts: int) -> np.ndarray:
    """Contiguous ranges of items balanced by weight (``kps_partition``)."""
    w = np.ascontiguousarray(weights, dtype=np.int64)
    bounds = np.zeros(parts + 1, dtype=np.int32)
    _check(lib().kps_partition(w.ctypes.data if len(w) else None, len(w), parts, bounds.ctypes.data))
    return bounds


class Turn:
    """A turn endgame (``kps_turn_*``): the turn round's folds and one river
    block per (turn ending, river card), run as one batched launch.  spec
    keys as synth.turn_spec: ranks, suits, cards_per_hand, board, stack,
    contrib0, bet_frac_t / raise_cap_t / allow_allin_t, bet_frac_r /
    raise_cap_r / allow_allin_r, mu1, mu2, strength [ranks*suits][H]."""

    def __init__(self, spec: dict):
        s = TurnSpec()
        s.ranks, s.suits = int(spec["ranks"]), int(spec["suits"])
        s.cards_per_hand = int(spec["cards_per_hand"])
        board = list(spec["board"])
        if len(board) > MAX_BOARD:
            raise ValueError("board too long")
        s.nboard = len(board)
        for i, c in enumerate(board):
            s.board[i] = int(c)
        s.stack[0], s.stack[1] = [float(v) for v in spec["stack"]]
        s.contrib0[0], s.contrib0[1] = [float(v) for v in spec["contrib0"]]
        for tag, name in (("t", "turn"), ("r", "river")):
            fr = list(spec["bet_frac_" + tag])
            if len(fr) > MAX_BETS:
                raise ValueError("too many bet sizes")
            setattr(s, "nbet_" + name, len(fr))
            arr = getattr(s, "bet_frac_" + name)
            for i, f in enumerate(fr):
                arr[i] = float(f)
            setattr(s, "raise_cap_" + name, int(spec["raise_cap_" + tag]))
            setattr(s, "allow_allin_" + name, 1 if spec.get("allow_allin_" + tag, False) else 0)
        self._strength = np.ascontiguousarray(spec["strength"], dtype=np.int32)
        mu1, mu2 = spec.get("mu1"), spec.get("mu2")
        self._mu1 = None if mu1 is None else np.ascontiguousarray(mu1, dtype=np.float64)
        self._mu2 = None if mu2 is None else np.ascontiguousarray(mu2, dtype=np.float64)
        s.strength = self._strength.ctypes.data_as(C.POINTER(C.c_int32))
        s.mu1 = self._mu1.ctypes.data_as(C.POINTER(C.c_double)) if self._mu1 is not None else None
        s.mu2 = self._mu2.ctypes.data_as(C.POINTER(C.c_double)) if self._mu2 is not None else None
        h = C.c_void_p()
        _check(lib().kps_turn_create(C.byref(s), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kps_turn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        v = np.zeros(9, dtype=np.int64)
        _check(lib().kps_turn_info(self._h, v.ctypes.data))
        keys = ("H", "hs", "n1", "n2", "endings", "blocks", "games", "turn_n1", "turn_n2")
        return {k: int(x) for k, x in zip(keys, v)}

    def offsets(self, player: int) -> np.ndarray:
        off = np.zeros(self.info()["games"] + 1, dtype=np.int64)
        _check(lib().kps_turn_offsets(self._h, int(player), off.ctypes.data))
        return off

    def block(self, i: int):
        """(ending, river card, canonical index of every hand position)."""
        e, r = C.c_int32(), C.c_int32()
        canon = np.zeros(self.info()["H"], dtype=np.int32)
        _check(lib().kps_turn_block(self._h, int(i), C.byref(e), C.byref(r), canon.ctypes.data))
        return e.value, r.value, canon

    def tune(self, dtype: int, stream=None) -> dict:
        """Autotune the launch shape of the batch behind the turn endgame."""
        b = C.c_void_p()
        _check(lib().kps_turn_batch(self._h, C.byref(b)))
        sh = BatchShape()
        _check(lib().kps_batch_tune(b, dtype, _stream(stream), C.byref(sh)))
        return sh.as_dict()

    def matvec_A(self, y, out, dtype=None, stream=None):
        _check(lib().kps_turn_matvec_A(self._h, _ptr(y), _ptr(out), _dtype_code(y, dtype), _stream(stream)))

    def matvec_AT(self, x, out, dtype=None, stream=None):
        _check(lib().kps_turn_matvec_AT(self._h, _ptr(x), _ptr(out), _dtype_code(x, dtype), _stream(stream)))


class Solver:
    """RM+ solver over a batch (``kps_solver_*``)."""

    def __init__(self, batch: Batch, dtype: int):
        self.batch = batch
        h = C.c_void_p()
        _check(lib().kps_solver_create(batch._h, dtype, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kps_solver_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, beh1=None, beh2=None, stream=None):
        _check(lib().kps_solver_reset(self._h, _ptr(beh1), _ptr(beh2), _stream(stream)))

    def warm_start(self, beh1, beh2, kappa: float, t0: int, stream=None):
        _check(lib().kps_solver_warm_start(self._h, _ptr(beh1), _ptr(beh2), float(kappa), int(t0), _stream(stream)))

    def set_method(self, method: int, alpha: float = 1.5, beta: float = 0.0, gamma: float = 2.0):
        """0 = RM+, 1 = Discounted CFR (takes effect at the next reset)."""
        _check(lib().kps_solver_set_method(self._h, int(method), float(alpha), float(beta), float(gamma)))

    def step(self, iters: int, stream=None):
        _check(lib().kps_solver_step(self._h, int(iters), _stream(stream)))

    def iterations(self) -> int:
        t = C.c_int64()
        _check(lib().kps_solver_iterations(self._h, C.byref(t)))
        return t.value

    def average(self, x, y, behavioural: bool = False, stream=None):
        _check(lib().kps_solver_average(self._h, 1 if behavioural else 0, _ptr(x), _ptr(y), _stream(stream)))

    def strategy(self, x, y, stream=None):
        _check(lib().kps_solver_strategy(self._h, _ptr(x), _ptr(y), _stream(stream)))

    def exploitability_estimate(self, expl, stream=None):
        _check(lib().kps_solver_exploitability_estimate(self._h, _ptr(expl), _stream(stream)))

    def exploitability(self, expl, br1=None, br2=None, stream=None):
        _check(lib().kps_solver_exploitability(self._h, _ptr(expl), _ptr(br1), _ptr(br2), _stream(stream)))

    def status(self):
        """kps_solver_status: raises KpsError(ENUMERIC) when the last step
        left a NaN or an infinity in the regrets or strategies."""
        _check(lib().kps_solver_status(self._h))

    def save(self, stream=None) -> bytes:
        """kps_solver_save: the solver's iteration state as bytes."""
        n = C.c_int64()
        _check(lib().kps_solver_state_bytes(self._h, C.byref(n)))
        buf = (C.c_ubyte * n.value)()
        _check(lib().kps_solver_save(self._h, C.cast(buf, C.c_void_p), n.value, _stream(stream)))
        return bytes(buf)

    def load(self, state: bytes, stream=None):
        """kps_solver_load: resume from bytes written by save()."""
        buf = (C.c_ubyte * len(state)).from_buffer_copy(state)
        _check(lib().kps_solver_load(self._h, C.cast(buf, C.c_void_p), len(state), _stream(stream)))


WARM_DIN = 1232
WARM_DOUT = 12


def warm_num_queries(batch: Batch) -> int:
    n = C.c_int64()
    _check(lib().kps_warm_num_queries(batch._h, C.byref(n)))
    return n.value


def warm_features(batch: Batch, X, nact=None, q0: int = 0, nq: int = None, qidx=None, stream=None):
    nq = len(qidx) if qidx is not None else nq
    _check(lib().kps_warm_features(batch._h, _ptr(qidx), int(q0), int(nq), _ptr(X), _ptr(nact), _stream(stream)))


def warm_targets(batch: Batch, beh1, beh2, x1, x2, T, w, q0: int = 0, nq: int = None, qidx=None, stream=None):
    nq = len(qidx) if qidx is not None else nq
    _check(lib().kps_warm_targets(batch._h, _ptr(beh1), _ptr(beh2), _ptr(x1), _ptr(x2), _ptr(qidx), int(q0),
                                  int(nq), _ptr(T), _ptr(w), _stream(stream)))


def warm_scatter(batch: Batch, P, beh1, beh2, q0: int = 0, nq: int = None, qidx=None, stream=None):
    nq = len(qidx) if qidx is not None else nq
    _check(lib().kps_warm_scatter(batch._h, _ptr(P), _ptr(qidx), int(q0), int(nq), _ptr(beh1), _ptr(beh2),
                                  _stream(stream)))


def warm_predict(batch: Batch, mlp: "MLP", beh1, beh2, stream=None):
    _check(lib().kps_warm_predict(batch._h, mlp._h, _ptr(beh1), _ptr(beh2), _stream(stream)))


class MLP:
    """The warm-start network (``kps_mlp_*``)."""

    def __init__(self, din: int = WARM_DIN, width: int = 256, dout: int = WARM_DOUT, seed: int = 0):
        h = C.c_void_p()
        _check(lib().kps_mlp_create(din, width, dout, seed, C.byref(h)))
        self._h = h
        self.din, self.width, self.dout = din, width, dout

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kps_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self) -> int:
        n = C.c_int64()
        _check(lib().kps_mlp_num_params(self._h, C.byref(n)))
        return n.value

    def get(self, which: int = 0) -> np.ndarray:
        out = np.zeros(self.num_params(), dtype=np.float32)
        _check(lib().kps_mlp_get(self._h, which, out.ctypes.data))
        return out

    def set(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().kps_mlp_set(self._h, p.ctypes.data))

    def forward(self, X, rows: int, nact, P, stream=None):
        _check(lib().kps_mlp_forward(self._h, _ptr(X), int(rows), _ptr(nact), _ptr(P), _stream(stream)))

    def gradients(self, X, rows: int, nact, T, w, wsum: float, loss=None, stream=None):
        _check(lib().kps_mlp_gradients(self._h, _ptr(X), int(rows), _ptr(nact), _ptr(T), _ptr(w), float(wsum),
                                       _ptr(loss), _stream(stream)))

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        _check(lib().kps_mlp_adam(self._h, lr, beta1, beta2, eps, _stream(stream)))

    def save(self) -> bytes:
        """kps_mlp_save: parameters, Adam moments and step count as bytes."""
        n = C.c_int64()
        _check(lib().kps_mlp_state_bytes(self._h, C.byref(n)))
        buf = (C.c_ubyte * n.value)()
        _check(lib().kps_mlp_save(self._h, C.cast(buf, C.c_void_p), n.value))
        return bytes(buf)

    def load(self, state: bytes):
        """kps_mlp_load: resume from bytes written by save()."""
        buf = (C.c_ubyte * len(state)).from_buffer_copy(state)
        _check(lib().kps_mlp_load(self._h, C.cast(buf, C.c_void_p), len(state)))


def version() -> str:
    return lib().kps_version().decode()
