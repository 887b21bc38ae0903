"""Python binding of libcountgauss: torch tensors in, torch tensors out.

PyTorch provides device memory and the current stream; every step of the transform
runs in the library's CUDA kernels, reached through the C ABI of
``include/countgauss.h``.  The functions here only check dtypes/devices, allocate
outputs and workspaces with torch, and pass pointers.

    plan = CountGauss(n, d, m, B, seed)
    Y = plan.apply_csr(row_ptr, col_idx, vals)   # G.(S.X), m x d   (Section 1.1)
    Y = plan.apply_dense(X)
    dX = plan.adjoint(dY)                        # S^T G^T dY
    Yp = plan.plain_csr(row_ptr, col_idx, vals)  # G~.X, the product it replaces
    Y = countgauss_dense(X, plan)                # differentiable (autograd)
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

_P = ctypes.c_void_p


def _ptr(t) -> _P:
    return _P(0) if t is None else _P(t.data_ptr())


def _stream(device) -> _P:
    return _P(torch.cuda.current_stream(device).cuda_stream)


def _need_host(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cpu":
        raise ValueError(f"{name} must be a CPU tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _need(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class CountGauss:
    """A CountGauss plan T = G.S for X of n rows and d columns (cg_plan_create).

    Calls run asynchronously on the current CUDA stream.  The calls made through one plan
    share its device workspace (one per device, grown on demand), so issue them on one
    stream, or synchronise between streams; use one plan per concurrent stream otherwise.
    Plans are host objects of a few bytes, and plans with the same seed, m and B apply the
    same T."""

    def __init__(self, n: int, d: int, m: int, B: int, seed: int, *, precision: str = "fp32",
                 deterministic: bool = False, row_offset: int = 0, ksplit: int = 0, sketch_ctas: int = 0,
                 scatter: str = "auto", scatter_passes: int = 0, scatter_rows: int = 0):
        lib = _lib.load()
        h = _P()
        _lib.check("cg_plan_create", lib.cg_plan_create(n, d, m, B, seed, ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.n, self.d, self.m, self.B, self.seed = int(n), int(d), int(m), int(B), int(seed)
        self._ws: dict = {}
        self.set_option(_lib.OPT_PRECISION, _lib.PREC[precision])
        self.set_option(_lib.OPT_DETERMINISTIC, int(bool(deterministic)))
        self.set_option(_lib.OPT_ROW_OFFSET, int(row_offset))
        self.set_option(_lib.OPT_KSPLIT, int(ksplit))
        self.set_option(_lib.OPT_SKETCH_CTAS, int(sketch_ctas))
        self.set_option(_lib.OPT_SCATTER, _lib.SCATTER[scatter])
        self.set_option(_lib.OPT_SCATTER_PASSES, int(scatter_passes))
        self.set_option(_lib.OPT_SCATTER_ROWS, int(scatter_rows))
        self.precision = precision
        self.deterministic = bool(deterministic)
        self.row_offset = int(row_offset)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.cg_plan_destroy(h)
            self._h = None

    # -- options and workspace ------------------------------------------------
    def set_option(self, option: int, value: int) -> None:
        _lib.check("cg_plan_set_option", self._lib.cg_plan_set_option(self._h, option, int(value)))
        self._ws.clear()

    def workspace_size(self, op: int, nnz: int = 0) -> int:
        sz = ctypes.c_size_t()
        _lib.check("cg_workspace_size", self._lib.cg_workspace_size(self._h, op, int(nnz), ctypes.byref(sz)))
        return int(sz.value)

    def workspace(self, op: int, nnz: int, device: torch.device) -> torch.Tensor:
        need = self.workspace_size(op, nnz)
        key = (device.index if device.index is not None else torch.cuda.current_device())
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
            ws[:256].zero_()  # status word starts clear
            self._ws[key] = ws
        return ws

    def enable_timing(self, on: bool = True) -> None:
        """Record CUDA events around each main kernel launch (CG_OPT_TIMING)."""
        _lib.check("cg_plan_set_option", self._lib.cg_plan_set_option(self._h, _lib.OPT_TIMING, int(bool(on))))

    def kernel_time(self, kernel: int):
        """(total ms, launches) of `kernel` since the last call (cg_plan_timing)."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _lib.check("cg_plan_timing", self._lib.cg_plan_timing(self._h, kernel, ctypes.byref(ms), ctypes.byref(n)))
        return float(ms.value), int(n.value)

    def check(self) -> None:
        """Synchronise and raise if any kernel since the last check set the status word."""
        for dev, ws in self._ws.items():
            _lib.check("cg_plan_check", self._lib.cg_plan_check(self._h, _ptr(ws), _stream(ws.device)))

    # -- the transform --------------------------------------------------------
    def apply_csr(self, row_ptr, col_idx, vals, out=None) -> torch.Tensor:
        """Y = G.(S.X) for CSR X (Section 1.1; Algorithm 1 steps 1-2).  row_ptr int32, or
        int64 for a matrix of 2^31 nonzeros or more (cg_apply_csr_i64)."""
        wide = torch.is_tensor(row_ptr) and row_ptr.dtype == torch.int64
        row_ptr = _need(row_ptr, torch.int64 if wide else torch.int32, "row_ptr")
        col_idx = _need(col_idx, torch.int32, "col_idx")
        vals = _need(vals, torch.float32, "vals")
        dev = row_ptr.device
        nnz = col_idx.numel()
        Y = torch.empty(self.m, self.d, dtype=torch.float32, device=dev) if out is None else out
        op, name = (_lib.OP_APPLY_CSR_I64, "cg_apply_csr_i64") if wide else (_lib.OP_APPLY_CSR, "cg_apply_csr")
        ws = self.workspace(op, nnz, dev)
        _lib.check(name, getattr(self._lib, name)(
            self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), nnz, _ptr(Y), _ptr(ws), ws.numel(), _stream(dev)))
        return Y

    def apply_right_csr(self, row_ptr, col_idx, vals, out=None) -> torch.Tensor:
        """Z = A.T^T (d x m) for a d x n CSR matrix A with one row per sample: the random
        projection X.R, R = T^T, of the SVM application (Section 9; Table 1)."""
        row_ptr = _need(row_ptr, torch.int32, "row_ptr")
        col_idx = _need(col_idx, torch.int32, "col_idx")
        vals = _need(vals, torch.float32, "vals")
        if row_ptr.numel() != self.d + 1:
            raise ValueError(f"row_ptr must have d + 1 = {self.d + 1} entries (one row per sample)")
        dev = row_ptr.device
        nnz = col_idx.numel()
        Z = torch.empty(self.d, self.m, dtype=torch.float32, device=dev) if out is None else out
        ws = self.workspace(_lib.OP_APPLY_RIGHT_CSR, nnz, dev)
        _lib.check("cg_apply_right_csr", self._lib.cg_apply_right_csr(
            self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), nnz, _ptr(Z), _ptr(ws), ws.numel(), _stream(dev)))
        return Z

    def apply_csr_host(self, row_ptr, col_idx, vals, out=None, device=None) -> torch.Tensor:
        """Y = G.(S.X) for a CSR X in host memory, Y returned in host memory
        (cg_apply_csr_host: chunked copies on a second stream overlap the scatter).
        Pinned CPU tensors make the copies asynchronous.  Synchronises the device's
        current stream before returning, so Y is ready."""
        row_ptr = _need_host(row_ptr, torch.int32, "row_ptr")
        col_idx = _need_host(col_idx, torch.int32, "col_idx")
        vals = _need_host(vals, torch.float32, "vals")
        if row_ptr.numel() != self.n + 1:
            raise ValueError(f"row_ptr must have n + 1 = {self.n + 1} entries")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        nnz = col_idx.numel()
        Y = torch.empty(self.m, self.d, dtype=torch.float32, pin_memory=True) if out is None else out
        if Y.device.type != "cpu" or not Y.is_contiguous() or Y.dtype != torch.float32:
            raise ValueError("out must be a contiguous float32 CPU tensor")
        ws = self.workspace(_lib.OP_APPLY_CSR_HOST, nnz, dev)
        _lib.check("cg_apply_csr_host", self._lib.cg_apply_csr_host(
            self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), nnz, _ptr(Y), _ptr(ws), ws.numel(), _stream(dev)))
        torch.cuda.current_stream(dev).synchronize()
        return Y

    def set_host_chunk(self, nnz_per_chunk: int) -> None:
        """Most nonzeros and rows per chunk of apply_csr_host (CG_OPT_HOST_CHUNK; 0: automatic)."""
        self.set_option(_lib.OPT_HOST_CHUNK, int(nnz_per_chunk))

    def set_host_read(self, mode: str) -> None:
        """How apply_csr_host gets the host CSR (CG_OPT_HOST_READ): "auto", "copied" (chunked
        copies by the copy engine) or "direct" (the scatter reads pinned host memory in place)."""
        self.set_option(_lib.OPT_HOST_READ, _lib.HOST_READ[mode])

    def apply_dense(self, X, out=None) -> torch.Tensor:
        """Y = G.(S.X) for dense row-major X (n x d)."""
        X = _need(X, torch.float32, "X")
        dev = X.device
        Y = torch.empty(self.m, self.d, dtype=torch.float32, device=dev) if out is None else out
        ws = self.workspace(_lib.OP_APPLY_DENSE, 0, dev)
        _lib.check("cg_apply_dense", self._lib.cg_apply_dense(
            self._h, _ptr(X), X.shape[1] if X.dim() == 2 else self.d, _ptr(Y), _ptr(ws), ws.numel(), _stream(dev)))
        return Y

    def adjoint(self, dY, row_ptr=None, col_idx=None, out=None) -> torch.Tensor:
        """dX = S^T.(G^T.dY): dense n x d, or nnz values at a CSR pattern (row_ptr int32,
        or int64 for 2^31 nonzeros or more: cg_apply_adjoint_i64)."""
        dY = _need(dY, torch.float32, "dY")
        dev = dY.device
        name = "cg_apply_adjoint"
        if row_ptr is None:
            dX = torch.empty(self.n, self.d, dtype=torch.float32, device=dev) if out is None else out
            nnz, op = 0, _lib.OP_ADJOINT_DENSE
        else:
            wide = torch.is_tensor(row_ptr) and row_ptr.dtype == torch.int64
            row_ptr = _need(row_ptr, torch.int64 if wide else torch.int32, "row_ptr")
            col_idx = _need(col_idx, torch.int32, "col_idx")
            nnz, op = col_idx.numel(), _lib.OP_ADJOINT_CSR
            name = "cg_apply_adjoint_i64" if wide else name
            dX = torch.empty(nnz, dtype=torch.float32, device=dev) if out is None else out
        ws = self.workspace(op, nnz, dev)
        _lib.check(name, getattr(self._lib, name)(
            self._h, _ptr(dY), _ptr(row_ptr), _ptr(col_idx), nnz, _ptr(dX), _ptr(ws), ws.numel(), _stream(dev)))
        return dX

    def plain_csr(self, row_ptr, col_idx, vals, out=None) -> torch.Tensor:
        """Y = G~.X with an on-the-fly m x n Gaussian (the product CountGauss replaces)."""
        row_ptr = _need(row_ptr, torch.int32, "row_ptr")
        col_idx = _need(col_idx, torch.int32, "col_idx")
        vals = _need(vals, torch.float32, "vals")
        dev = row_ptr.device
        nnz = col_idx.numel()
        Y = torch.empty(self.m, self.d, dtype=torch.float32, device=dev) if out is None else out
        ws = self.workspace(_lib.OP_PLAIN_CSR, nnz, dev)
        _lib.check("cg_plain_gaussian_apply", self._lib.cg_plain_gaussian_apply(
            self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), nnz, _ptr(Y), _ptr(ws), ws.numel(), _stream(dev)))
        return Y

    def nmf_anchors(self, row_ptr, col_idx, vals):
        """Algorithm 1 steps 1-3: Z = T.X and, per row of Z, the column of its max and
        of its min (lowest index on ties), taken inside the split-K sum.  Returns
        (Z, imax, imin).  int64 row_ptr (2^31 nonzeros or more) runs
        cg_nmf_anchors_csr_i64."""
        wide = torch.is_tensor(row_ptr) and row_ptr.dtype == torch.int64
        row_ptr = _need(row_ptr, torch.int64 if wide else torch.int32, "row_ptr")
        col_idx = _need(col_idx, torch.int32, "col_idx")
        vals = _need(vals, torch.float32, "vals")
        dev = row_ptr.device
        nnz = col_idx.numel()
        Z = torch.empty(self.m, self.d, dtype=torch.float32, device=dev)
        imax = torch.empty(self.m, dtype=torch.int32, device=dev)
        imin = torch.empty(self.m, dtype=torch.int32, device=dev)
        ws = self.workspace(_lib.OP_APPLY_CSR_I64 if wide else _lib.OP_APPLY_CSR, nnz, dev)
        name = "cg_nmf_anchors_csr_i64" if wide else "cg_nmf_anchors_csr"
        _lib.check(name, getattr(self._lib, name)(
            self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), nnz, _ptr(Z), _ptr(imax), _ptr(imin), _ptr(ws),
            ws.numel(), _stream(dev)))
        return Z, imax, imin

    # -- stages -----------------------------------------------------------------
    def _sketch_out(self, out, accumulate: bool, dev) -> torch.Tensor:
        if accumulate and out is None:
            raise ValueError("accumulate=True needs out=SX to add into")
        if out is not None and (out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != self.B * self.d):
            raise ValueError(f"out must be a contiguous float32 tensor of B x d = {self.B} x {self.d}")
        self.set_option(_lib.OPT_ACCUMULATE, int(bool(accumulate)))
        return torch.empty(self.B, self.d, dtype=torch.float32, device=dev) if out is None else out

    def sketch_csr(self, row_ptr, col_idx, vals, out=None, accumulate: bool = False) -> torch.Tensor:
        """SX = S.X (Section 1.1), or SX += S.X into `out` with accumulate=True: rows of X fed
        in chunks (each with its global row offset, set_row_offset) sketch into one SX, and a
        saved SX plus the next row offset resumes the stream.  row_ptr int32, or int64 for
        2^31 nonzeros or more (cg_sketch_csr_i64)."""
        wide = torch.is_tensor(row_ptr) and row_ptr.dtype == torch.int64
        row_ptr = _need(row_ptr, torch.int64 if wide else torch.int32, "row_ptr")
        col_idx = _need(col_idx, torch.int32, "col_idx")
        vals = _need(vals, torch.float32, "vals")
        dev = row_ptr.device
        nnz = col_idx.numel()
        SX = self._sketch_out(out, accumulate, dev)
        op, name = (_lib.OP_SKETCH_I64, "cg_sketch_csr_i64") if wide else (_lib.OP_SKETCH, "cg_sketch_csr")
        ws = self.workspace(op, nnz, dev)
        _lib.check(name, getattr(self._lib, name)(
            self._h, _ptr(row_ptr), _ptr(col_idx), _ptr(vals), nnz, _ptr(SX), _ptr(ws), ws.numel(), _stream(dev)))
        return SX

    def sketch_dense(self, X, out=None, accumulate: bool = False) -> torch.Tensor:
        """SX = S.X for dense X, or SX += S.X into `out` with accumulate=True."""
        X = _need(X, torch.float32, "X")
        dev = X.device
        SX = self._sketch_out(out, accumulate, dev)
        ws = self.workspace(_lib.OP_SKETCH, 0, dev)
        _lib.check("cg_sketch_dense", self._lib.cg_sketch_dense(
            self._h, _ptr(X), X.shape[1], _ptr(SX), _ptr(ws), ws.numel(), _stream(dev)))
        return SX

    def set_row_offset(self, row_offset: int) -> None:
        """Global index of local row 0 (CG_OPT_ROW_OFFSET), e.g. per chunk of a stream."""
        self.set_option(_lib.OPT_ROW_OFFSET, int(row_offset))
        self.row_offset = int(row_offset)

    def contract(self, SX, out=None) -> torch.Tensor:
        SX = _need(SX, torch.float32, "SX")
        dev = SX.device
        Y = torch.empty(self.m, self.d, dtype=torch.float32, device=dev) if out is None else out
        ws = self.workspace(_lib.OP_CONTRACT, 0, dev)
        _lib.check("cg_contract", self._lib.cg_contract(
            self._h, _ptr(SX), _ptr(Y), _ptr(ws), ws.numel(), _stream(dev)))
        return Y


# -- batches -----------------------------------------------------------------------
class CountGaussBatch:
    """Many instances in one persistent launch (cg_batch_plan_create / cg_batch_apply).

    `instances` is a list of dicts with keys n, d, m, B, seed, row_ptr, col_idx, vals
    (CUDA tensors: int32, int32, float32).  Outputs are allocated here (self.Y[k], m x d);
    the tensors are kept alive by this object, since the plan holds their pointers."""

    def __init__(self, instances, *, graph: bool = True, wait_us: int | None = None):
        lib = _lib.load()
        self._lib = lib
        self._keep = []
        self.Y = []
        descs = (_lib.BatchDesc * len(instances))()
        dev = None
        for k, inst in enumerate(instances):
            rp = _need(inst["row_ptr"], torch.int32, "row_ptr")
            ci = _need(inst["col_idx"], torch.int32, "col_idx")
            v = _need(inst["vals"], torch.float32, "vals")
            dev = rp.device
            Y = torch.empty(inst["m"], inst["d"], dtype=torch.float32, device=dev)
            self._keep += [rp, ci, v]
            self.Y.append(Y)
            descs[k] = _lib.BatchDesc(inst["n"], inst["d"], inst["m"], inst["B"], inst["seed"], rp.data_ptr(),
                                      ci.data_ptr(), v.data_ptr(), ci.numel(), Y.data_ptr())
        self.device = dev if dev is not None else torch.device("cuda")
        h = _P()
        _lib.check("cg_batch_plan_create",
                   lib.cg_batch_plan_create(ctypes.cast(descs, _P), len(instances), ctypes.byref(h)))
        self._h = h
        self.set_option(_lib.BATCH_OPT_GRAPH, int(bool(graph)))
        if wait_us is not None:
            self.set_option(_lib.BATCH_OPT_WAIT_US, int(wait_us))
        self._ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.cg_batch_plan_destroy(h)
            self._h = None

    def set_option(self, option: int, value: int) -> None:
        _lib.check("cg_batch_set_option", self._lib.cg_batch_set_option(self._h, option, int(value)))

    def get_option(self, option: int) -> int:
        v = ctypes.c_int64()
        _lib.check("cg_batch_plan_get_option", self._lib.cg_batch_plan_get_option(self._h, option, ctypes.byref(v)))
        return int(v.value)

    def workspace(self) -> torch.Tensor:
        sz = ctypes.c_size_t()
        _lib.check("cg_batch_workspace_size", self._lib.cg_batch_workspace_size(self._h, ctypes.byref(sz)))
        if self._ws is None or self._ws.numel() < sz.value:
            self._ws = torch.empty(max(int(sz.value), 256), dtype=torch.uint8, device=self.device)
            self._ws[:256].zero_()
        return self._ws

    def apply(self):
        ws = self.workspace()
        _lib.check("cg_batch_apply", self._lib.cg_batch_apply(self._h, _ptr(ws), ws.numel(), _stream(self.device)))
        return self.Y

    def check(self) -> None:
        ws = self.workspace()
        _lib.check("cg_batch_check", self._lib.cg_batch_check(self._h, _ptr(ws), _stream(self.device)))

    def autotune(self, reps: int = 3) -> float:
        ws = self.workspace()
        best = ctypes.c_double()
        _lib.check("cg_batch_autotune", self._lib.cg_batch_autotune(self._h, _ptr(ws), ws.numel(),
                                                                    _stream(self.device), reps, ctypes.byref(best)))
        return float(best.value)


# -- distribution checker -------------------------------------------------------------
def moments_f64(Y: torch.Tensor, gram: torch.Tensor | None = None, sumsq: torch.Tensor | None = None):
    """gram += Y^T Y and sumsq += ||Y||_F^2 in FP64 on the device (cg_moments_f64).
    Y: CUDA float32 (rows, d).  New zeroed accumulators are made when not given."""
    Y = _need(Y, torch.float32, "Y")
    d = Y.shape[1]
    if gram is None:
        gram = torch.zeros(d, d, dtype=torch.float64, device=Y.device)
    if sumsq is None:
        sumsq = torch.zeros(1, dtype=torch.float64, device=Y.device)
    _lib.call("cg_moments_f64", _ptr(Y), Y.shape[0], d, _ptr(gram), _ptr(sumsq), _stream(Y.device))
    return gram, sumsq


def row_argmax_argmin(Z: torch.Tensor):
    """Algorithm 1 step 3 on a device matrix Z (m x d): (imax, imin), int32."""
    Z = _need(Z, torch.float32, "Z")
    m, d = Z.shape
    imax = torch.empty(m, dtype=torch.int32, device=Z.device)
    imin = torch.empty(m, dtype=torch.int32, device=Z.device)
    _lib.call("cg_row_argmax_argmin", _ptr(Z), m, d, _ptr(imax), _ptr(imin), _stream(Z.device))
    return imax, imin


# -- generator dumps (bit-exact checks against the oracle) -----------------------
def generate_words(seed: int, tag: int, idx0: int, count: int, device="cuda") -> torch.Tensor:
    out = torch.empty(count, 4, dtype=torch.int32, device=device)
    _lib.call("cg_generate_words", seed, tag, idx0, count, _ptr(out), _stream(out.device))
    return out


def generate_hash_sign(seed: int, B: int, row0: int, count: int, device="cuda"):
    h = torch.empty(count, dtype=torch.int32, device=device)
    s = torch.empty(count, dtype=torch.int32, device=device)
    _lib.call("cg_generate_hash_sign", seed, B, row0, count, _ptr(h), _ptr(s), _stream(h.device))
    return h, s


def generate_gaussian(seed: int, tag: int, R: int, r0: int, r1: int, c0: int, c1: int, device="cuda"):
    out = torch.empty(r1 - r0, c1 - c0, dtype=torch.float32, device=device)
    _lib.call("cg_generate_gaussian", seed, tag, R, r0, r1, c0, c1, _ptr(out), _stream(out.device))
    return out


def diag_random_reductions(array, count: int):
    """Add 1.0 at `count` hashed positions of the float32 device tensor `array`
    (cg_diag_random_reductions: the reduction-rate ceiling of the scatter)."""
    array = _need(array, torch.float32, "array")
    _lib.call("cg_diag_random_reductions", _ptr(array), array.numel(), int(count), _stream(array.device))
    return array


# -- autograd ---------------------------------------------------------------------
class CountGaussDenseFn(torch.autograd.Function):
    """Y = T.X for dense X; backward dX = T^T dY = S^T (G^T dY) with G regenerated."""

    @staticmethod
    def forward(ctx, X, plan):
        ctx.plan = plan
        return plan.apply_dense(X.contiguous())

    @staticmethod
    def backward(ctx, dY):
        return ctx.plan.adjoint(dY.contiguous()), None


class CountGaussCsrFn(torch.autograd.Function):
    """Y = T.X for CSR X as a function of its stored values; backward is the
    gradient at the stored entries only."""

    @staticmethod
    def forward(ctx, vals, row_ptr, col_idx, plan):
        ctx.plan = plan
        ctx.save_for_backward(row_ptr, col_idx)
        return plan.apply_csr(row_ptr, col_idx, vals.contiguous())

    @staticmethod
    def backward(ctx, dY):
        row_ptr, col_idx = ctx.saved_tensors
        return ctx.plan.adjoint(dY.contiguous(), row_ptr, col_idx), None, None, None


def countgauss_dense(X: torch.Tensor, plan: CountGauss) -> torch.Tensor:
    return CountGaussDenseFn.apply(X, plan)


def countgauss_csr(vals: torch.Tensor, row_ptr: torch.Tensor, col_idx: torch.Tensor, plan: CountGauss) -> torch.Tensor:
    return CountGaussCsrFn.apply(vals, row_ptr, col_idx, plan)
