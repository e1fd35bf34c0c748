"""Continuous-batching server of dd SPD solves: F = Rsyrk(G), Rpotrf(F), Rpotrs.

Each request brings G (n x 2n) and B (n x nrhs) as dd matrices.  Its work is
a fixed list of operations on its own device buffers:

  * F := G G^T: for n >= ``sliced_min_n`` one split-precision Rsyrk on the
    tensor cores (``mp_dd_Rsyrk_crt``, the residue form, upper triangle,
    within the same accuracy bound); for smaller n one FP64 Rsyrk-type
    update of the upper triangle;
  * the blocked Cholesky F = U^T U in groups of ``group`` blocks of 64
    columns: per block J of a group the update of its row block by the
    group's earlier blocks (F(J, J:) -= U(G0:J, J)^T U(G0:J, J:), left-looking,
    depth up to 192), the diagonal factorisation and the panel solve
    U_JJ^T X = F(J, J+1:); after the group, one update of the trailing
    matrix by the whole group (depth 256, upper triangle).  Updates of
    ``crt_min_rest`` columns or more run in residue form on the tensor cores
    (``mp_dd_Rgemm_crt`` / ``mp_dd_Rsyrk_crt``), within the same accuracy
    bound and far faster (a 2048 x 2048 x 256 update: 0.4 ms against ~13 ms
    in FP64); the residue form's cost is mostly per output entry, so one
    depth-256 trailing update costs about what one of depth 64 does;
  * the solve F X = B: blocked forward (U^T) and backward (U) substitution.

A scheduler step takes the next step of every admitted request -- a short
list of operations, e.g. a block's trailing update, diagonal factor and panel
solve -- and runs all of them in a fixed launch order: tensor-core products,
one grouped dd Rgemm launch for every Rsyrk/Rgemm-type operation
(``mp_dd_Rgemm_grouped``), one batched diagonal factorisation
(``mp_dd_potrf_diag_batch``) and one batched triangular solve
(``mp_dd_trsm_batch``).  A request of order n takes about 2 n / 64 steps:
the Cholesky blocks with the forward substitution one block behind, then
the backward substitution.  Requests arriving while others run are admitted as
soon as a slot and device memory (the budget) are free, and join the next
step.  A request's operation sequence and every operation's arithmetic are
independent of which other requests share the step, so each result is
bitwise the same alone and in the mix.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import (_abi, mp_dd_potrf_diag_batch, mp_dd_Rgemm_crt, mp_dd_Rgemm_crt_workspace,
               mp_dd_Rsyrk_crt, mp_dd_Rsyrk_crt_workspace, mp_dd_trsm_batch, to_device,
               to_numpy, workspace)
from . import grouped as gr


@dataclass
class Request:
    rid: int
    n: int
    G: tuple | None     # (hi, lo) n x 2n, column-major: numpy (host) or torch (device)
    B: tuple | None     # (hi, lo) n x nrhs
    arrival: float = 0.0
    nrhs_: int = 4
    loader: object = None   # callable returning (G, B) at admission, when G is None
    # filled in by the server
    admit_t: float = 0.0
    done_t: float = 0.0
    ops: list = field(default_factory=list)   # steps, each a list of operations
    pos: int = 0
    dev: dict = field(default_factory=dict)
    X: tuple | None = None
    info: int = 0

    @property
    def nrhs(self) -> int:
        return int(self.B[0].shape[1]) if self.B is not None else self.nrhs_

    sliced_ws: int = 0    # workspace bytes of the tensor-core Rsyrk (0 = FP64 path)

    def footprint(self) -> int:
        """Device bytes while admitted: G, F, X planes, the info word and the
        sliced-Rsyrk workspace when that path is used."""
        n = self.n
        return 16 * (2 * n * n + n * n + n * self.nrhs) + 64 + self.sliced_ws

    def flops(self) -> float:
        """dd operation count: Rsyrk k n (n+1) with k = 2n, Rpotrf n^3/3,
        Rpotrs 2 n^2 nrhs (the LAPACK counts)."""
        n = float(self.n)
        return 2 * n * n * (n + 1) + n ** 3 / 3 + 2 * n * n * self.nrhs


def _view(P, r0, c0, rows, cols):
    return P[r0:r0 + rows, c0:c0 + cols]


def _pair(D, r0, c0, rows, cols):
    return (_view(D[0], r0, c0, rows, cols), _view(D[1], r0, c0, rows, cols))


class SpdServer:
    """Admission, per-request operation lists and the batched scheduler step."""

    def __init__(self, budget_bytes: float = 120e9, slots: int = 256, nb: int = 64,
                 table: dict | None = None, sliced_min_n: int = 256, crt_min_rest: int = 512,
                 depth: int = 2, group: int = 4):
        self.sliced_min_n = int(sliced_min_n)
        self.crt_min_rest = int(crt_min_rest)
        self.group = max(1, int(group))
        self.budget = float(budget_bytes)
        self.slots = int(slots)
        self.nb = int(nb)
        self.table = table
        self.active: list[Request] = []
        self.draining: list = []    # finished on the device, result copy in flight
        self.inflight: list = []    # events of the steps queued on the GPU
        self.depth = int(depth)
        self.used = 0
        self.steps = 0
        self.max_active = 0
        self.launches = 0

    # ---------------------------------------------------------------- admission

    def can_admit(self, r: Request) -> bool:
        self._size(r)
        return (len(self.active) < self.slots
                and self.used + r.footprint() <= self.budget)

    def _size(self, r: Request) -> None:
        if r.n >= self.sliced_min_n and r.sliced_ws == 0:
            # one workspace for F = G G^T (k = 2n), the group updates (k =
            # group nb) and the row-block updates (nb rows, k < group nb)
            kg = self.group * self.nb
            r.sliced_ws = max(mp_dd_Rsyrk_crt_workspace(r.n, 2 * r.n),
                              mp_dd_Rsyrk_crt_workspace(r.n, kg),
                              mp_dd_Rgemm_crt_workspace(self.nb, r.n, max(1, kg - self.nb)))

    def admit(self, r: Request, now: float) -> None:
        self._size(r)
        n, nrhs = r.n, r.nrhs
        Gs, Bs = (r.G, r.B) if r.G is not None else r.loader()
        G = tuple(x if isinstance(x, torch.Tensor) else to_device(x) for x in Gs)
        F = tuple(torch.zeros((n, n), dtype=torch.float64, device="cuda").t()
                  for _ in range(2))
        X = tuple(x.clone() if isinstance(x, torch.Tensor) else to_device(x) for x in Bs)
        info = torch.zeros(1, dtype=torch.int64, device="cuda")
        r.dev = {"G": G, "F": F, "X": X, "info": info}
        if r.sliced_ws:
            r.dev["ws"] = workspace(r.sliced_ws)
        r.ops = self._compile(r, self._plan(r))
        r.pos = 0
        r.admit_t = now
        self.active.append(r)
        self.used += r.footprint()
        self.max_active = max(self.max_active, len(self.active))

    def _plan(self, r: Request) -> list:
        """The request's steps, each a list of operations that run in the same
        scheduler step.  A step's launches run in a fixed order -- tensor-core
        products (at collection), then the grouped FP64 Rgemm, the batched
        diagonal factorisations, the batched triangular solves -- so one step
        can hold a block's dependent chain: the trailing update left by the
        previous block, then this block's diagonal factor and panel solve
        (likewise the update and the block solve of the substitutions)."""
        n, nrhs, nb = r.n, r.nrhs, self.nb
        G, F, X = r.dev["G"], r.dev["F"], r.dev["X"]
        one, mone, zero = (1.0, 0.0), (-1.0, 0.0), (0.0, 0.0)
        steps = []
        # F := G G^T: the tensor-core product, or below sliced_min_n one FP64
        # Rsyrk-type update of the upper triangle (k = 2n < 512, a small
        # share of a step)
        if r.sliced_ws:
            steps.append([("sliced", (G, F))])
        else:
            steps.append([("gemm", ("N", "T", n, n, 2 * n, one, G, G, zero, F, 1))])
        # blocked Cholesky, upper, in groups of `group` blocks: block J's
        # step = [the group update left by the previous group (first block
        # of a group) or the row-block update by the group's earlier blocks,
        # diagonal factor J, panel solve J]; the first joins the F step.
        # The forward substitution U^T Y = B runs one block behind in the same
        # steps: block J's solve needs only U_JJ and the updates from blocks
        # before it, and its update of the later rows only the finished row
        # block U(J, J+1:), so step J also holds [forward update left by
        # J-2, forward solve J-1] (the grouped launch runs before the
        # triangular solves).  The last forward pair follows the loop.
        blocks = list(range(0, n, nb))
        fwd_trsm, fwd_upd = [], []
        for j in blocks:
            b = min(nb, n - j)
            fwd_trsm.append(("trsm", (_pair(F, j, j, b, b), _pair(X, j, 0, b, nrhs), b, nrhs, 1)))
            rest = n - j - b
            fwd_upd.append(("gemm", ("T", "N", rest, nrhs, b, mone, _pair(F, j, j + b, b, rest),
                                     _pair(X, j, 0, b, nrhs), one,
                                     _pair(X, j + b, 0, rest, nrhs), 0)) if rest > 0 else None)
        crt_ok = bool(r.sliced_ws)
        pending = None
        for t, j in enumerate(blocks):
            b = min(nb, n - j)
            g0 = (t // self.group) * self.group * nb          # the group's first column
            ops = [pending] if pending else []
            pending = None
            if j > g0:
                # F(J, J:) -= U(g0:J, J)^T U(g0:J, J:), depth j - g0
                cols, k = n - j, j - g0
                Ut, Pr, Cr = _pair(F, g0, j, k, b), _pair(F, g0, j, k, cols), _pair(F, j, j, b, cols)
                if crt_ok and cols >= self.crt_min_rest:
                    ops.append(("crt_gemm", (Ut, Pr, Cr, b, cols, k)))
                else:
                    ops.append(("gemm", ("T", "N", b, cols, k, mone, Ut, Pr, one, Cr, 0)))
            ops.append(("diag", (_pair(F, j, j, b, b), b, j)))
            rest = n - j - b
            if rest > 0:
                ops.append(("trsm", (_pair(F, j, j, b, b), _pair(F, j, j + b, b, rest), b,
                                     rest, 1)))
                if t % self.group == self.group - 1:
                    # the group is done: F(e:, e:) -= U(g0:e, e:)^T U(g0:e, e:)
                    e, kg = j + b, j + b - g0
                    P, Ct = _pair(F, g0, e, kg, rest), _pair(F, e, e, rest, rest)
                    if crt_ok and rest >= self.crt_min_rest:
                        pending = ("crt", (P, Ct, rest, kg))
                    else:
                        pending = ("gemm", ("T", "N", rest, rest, kg, mone, P, P, one, Ct, 1))
            if t >= 2 and fwd_upd[t - 2]:
                ops.append(fwd_upd[t - 2])
            if t >= 1:
                ops.append(fwd_trsm[t - 1])
            if t == 0:
                steps[-1].extend(ops)
            else:
                steps.append(ops)
        last = len(blocks) - 1
        if last == 0:
            steps[-1].append(fwd_trsm[0])      # after its diagonal factor in launch order
        else:
            steps.append(([fwd_upd[last - 1]] if fwd_upd[last - 1] else []) + [fwd_trsm[last]])
        # backward substitution U X = Y, last block first (its own step: the
        # forward solve of the same block is in the previous one)
        pending = None
        for j in reversed(range(0, n, nb)):
            b = min(nb, n - j)
            ops = [pending] if pending else []
            ops.append(("trsm", (_pair(F, j, j, b, b), _pair(X, j, 0, b, nrhs), b, nrhs, 0)))
            pending = None
            if j > 0:
                pending = ("gemm", ("N", "N", j, nrhs, b, mone, _pair(F, 0, j, j, b),
                                    _pair(X, j, 0, b, nrhs), one, _pair(X, 0, 0, j, nrhs), 0))
            steps.append(ops)
        return steps

    def _compile(self, r: Request, steps: list) -> list:
        """Turn every batched operation into its descriptor bytes once, at
        admission (the pointers and sizes never change), so that a scheduler
        step only concatenates bytes."""
        info = r.dev["info"]
        out = []
        for ops in steps:
            cops = []
            for kind, args in ops:
                if kind == "gemm":
                    ta, tb, m, n, k, al, A, B, be, C, uplo = args
                    d = gr.desc(ta, tb, m, n, k, al, A, B, be, C, gr.shape_for(self.table, m, n),
                                uplo, info)
                    cops.append(("gemm", bytes(d)))
                elif kind == "diag":
                    P, b, off = args
                    d = _abi.MpDDPotrfDiagDesc()
                    d.a_hi, d.a_lo = P[0].data_ptr(), P[1].data_ptr()
                    d.lda, d.n, d.offset = P[0].stride(1), b, off
                    d.info, d.lower = info.data_ptr(), 0
                    cops.append(("diag", bytes(d)))
                elif kind == "trsm":
                    U, Bm, b, cols, trans = args
                    d = _abi.MpDDTrsmDesc()
                    d.u_hi, d.u_lo, d.ldu = U[0].data_ptr(), U[1].data_ptr(), U[0].stride(1)
                    d.b_hi, d.b_lo = Bm[0].data_ptr(), Bm[1].data_ptr()
                    d.ldb = max(Bm[0].stride(1), Bm[0].shape[0])
                    d.n, d.nrhs, d.info = b, cols, info.data_ptr()
                    d.trans, d.lower_u, d.lower_b = trans, 0, 0
                    cops.append(("trsm", (bytes(d), cols)))
                else:
                    cops.append((kind, args))
            out.append(cops)
        return out

    # ---------------------------------------------------------------- one step

    def step(self) -> list[Request]:
        """Run the next step of every active request.  Requests whose last
        step this was start an asynchronous copy of X to the host; returns the
        requests whose copies have landed (finished, results on the host)."""
        gemm, diag, trsm = [], [], []
        max_rhs = 0
        for r in self.active:
            for kind, args in r.ops[r.pos]:
                if kind == "gemm":
                    gemm.append(args)
                elif kind == "diag":
                    diag.append(args)
                elif kind == "trsm":
                    trsm.append(args[0])
                    max_rhs = max(max_rhs, args[1])
                elif kind == "sliced":
                    G, F = args
                    n = r.n
                    ws = r.dev["ws"]
                    mp_dd_Rsyrk_crt("U", "N", n, 2 * n, (1.0, 0.0), G, n, (0.0, 0.0), F, n, ws,
                                    ws.numel())
                    self.launches += 1
                elif kind == "crt":
                    P, Ct, rest, b = args
                    ws = r.dev["ws"]
                    mp_dd_Rsyrk_crt("U", "T", rest, b, (-1.0, 0.0), P, P[0].stride(1),
                                    (1.0, 0.0), Ct, Ct[0].stride(1), ws, ws.numel())
                    self.launches += 1
                else:   # "crt_gemm": a row block's update by its group's earlier blocks
                    Ut, Pr, Cr, b, cols, k = args
                    ws = r.dev["ws"]
                    ld = Cr[0].stride(1)
                    mp_dd_Rgemm_crt("T", "N", b, cols, k, (-1.0, 0.0), Ut, ld, Pr, ld, (1.0, 0.0),
                                    Cr, ld, ws, ws.numel())
                    self.launches += 1
        if gemm:
            arr = (_abi.MpDDGemmDesc * len(gemm)).from_buffer_copy(b"".join(gemm))
            ws = workspace(gr.mp_dd_Rgemm_grouped_workspace(len(arr), arr))
            gr.mp_dd_Rgemm_grouped_prepare(len(arr), arr, ws, ws.numel())
            gr.mp_dd_Rgemm_grouped_run(ws)
            self.launches += 1
        if diag:
            mp_dd_potrf_diag_batch(len(diag), _to_device_bytes(b"".join(diag)))
            self.launches += 1
        if trsm:
            mp_dd_trsm_batch(len(trsm), _to_device_bytes(b"".join(trsm)), max_rhs)
            self.launches += 1
        still = []
        for r in self.active:
            r.pos += 1
            if r.pos < len(r.ops):
                still.append(r)
                continue
            # done on the device: copy X and info out without stopping the GPU
            Xh = tuple(torch.empty(x.shape[::-1], dtype=x.dtype, pin_memory=True)
                       for x in r.dev["X"])
            for h, x in zip(Xh, r.dev["X"]):
                h.copy_(x.t(), non_blocking=True)
            ih = torch.empty(1, dtype=torch.int64, pin_memory=True)
            ih.copy_(r.dev["info"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record()
            self.draining.append((r, Xh, ih, ev))
        self.active = still
        self.steps += 1
        # keep at most `depth` steps queued on the GPU: the host prepares the
        # next step while the GPU runs the previous one, but a new arrival
        # never queues behind a long backlog of launched steps
        ev = torch.cuda.Event()
        ev.record()
        self.inflight.append(ev)
        while len(self.inflight) > self.depth:
            self.inflight.pop(0).synchronize()
        return self._harvest()

    def _harvest(self, wait: bool = False) -> list[Request]:
        """Requests whose result copies have completed (all of them with wait)."""
        done, keep = [], []
        for item in self.draining:
            r, Xh, ih, ev = item
            if wait:
                ev.synchronize()
            elif not ev.query():
                keep.append(item)
                continue
            r.done_t = time.perf_counter()
            r.X = (Xh[0].numpy().T, Xh[1].numpy().T)
            r.info = int(ih.item())
            self.used -= r.footprint()
            r.dev = {}
            done.append(r)
        self.draining = keep
        return done

    # ---------------------------------------------------------------- driver

    def serve(self, requests: list[Request], time_scale: float = 1.0) -> list[Request]:
        """Serve requests arriving at r.arrival seconds (relative to the start):
        admit whatever has arrived and fits, run a step, repeat.  Returns the
        requests in completion order with admit/done times on the same clock."""
        pending = sorted(requests, key=lambda r: r.arrival)
        done: list[Request] = []
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or self.active or self.draining:
            now = time.perf_counter() - t0
            if i < len(pending) and pending[i].footprint() > self.budget:
                raise ValueError(f"request {pending[i].rid} needs more than the memory budget")
            while i < len(pending) and pending[i].arrival * time_scale <= now and \
                    self.can_admit(pending[i]):
                self.admit(pending[i], now)
                i += 1
            if self.active:
                finished = self.step()
            else:
                # nothing to launch: collect results, wait for arrivals or copies
                finished = self._harvest(wait=i >= len(pending))
                if not finished and i < len(pending):
                    time.sleep(max(0.0, min(0.0005, pending[i].arrival * time_scale - now)))
            for r in finished:
                r.done_t -= t0
                done.append(r)
        return done


def _to_device_bytes(data: bytes) -> torch.Tensor:
    """Descriptor bytes on the device without waiting for the GPU: staged in
    pinned memory (PyTorch's host allocator keeps the block until the copy is
    done) and copied asynchronously on the current stream."""
    host = torch.frombuffer(bytearray(data), dtype=torch.uint8).pin_memory()
    return host.to("cuda", non_blocking=True)


def residual_ratio(F_host, X_host, B_host, mp) -> float:
    """LAPACK test ratio ||B - F X||_1 / (||F||_1 ||X||_1 eps_dd) with the
    residual computed by the library's dd Rgemm on the device (F symmetric,
    both triangles given)."""
    Fd = tuple(to_device(x) for x in F_host)
    Xd = tuple(to_device(x) for x in X_host)
    Rd = tuple(to_device(x) for x in B_host)
    n, nrhs = F_host[0].shape[0], X_host[0].shape[1]
    mp.mp_dd_Rgemm("N", "N", n, nrhs, n, (-1.0, 0.0), Fd, n, Xd, n, (1.0, 0.0), Rd, n)
    torch.cuda.synchronize()
    R = mp.to_numpy(Rd[0]) + mp.to_numpy(Rd[1])
    fn = np.abs(F_host[0]).sum(axis=0).max()
    xn = np.abs(X_host[0]).sum(axis=0).max()
    return float(np.abs(R).sum(axis=0).max() / (fn * xn * 2.0 ** -104))
