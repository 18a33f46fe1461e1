"""Python binding of libqhap (ctypes).  Argument marshalling only: every step of the
phasing path runs in the library's CUDA kernels.

The raw C functions are exposed under their C names (``qh_create``, ``qh_build_graph``,
``qh_bsb_solve``, ``qh_phase`` ...) through :func:`lib`.  The classes below wrap them
with numpy / torch arrays:

    ctx = Context(device=0)
    g = ctx.build_graph(frags, mode=MODE_READ, weight_mode=WEIGHT_SIGNED)
    sol = ctx.solve(g, replicas=1024, steps=1000, precision=PREC_BF16, seed=1)
    hap1, hap2, block_id = ctx.phase(g, sol)

Importing succeeds without a GPU; creating a Context needs the CUDA library
(``libqhap.so``, built by ``paper_2603_25762_gb300.build.build()``) and raises if it
is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("QHAP_LIB") or os.path.join(HERE, "libqhap.so")

QH_OK, QH_EINVAL, QH_ENOMEM, QH_ECUDA, QH_ETIMEOUT, QH_EUNSUPPORTED = range(6)
MODE_READ, MODE_SNP = 0, 1
WEIGHT_CONFLICT, WEIGHT_SIGNED = 0, 1
PREC_FP32, PREC_BF16, PREC_BF16X2, PREC_FP8 = 0, 1, 2, 3
SCHED_LINEAR, SCHED_AUTO = 0, 1
STORAGE_AUTO, STORAGE_TILES, STORAGE_CSR = 0, 1, 2


class QhFragments(C.Structure):
    _fields_ = [("n_frags", C.c_int32), ("n_snps", C.c_int32), ("frag_ptr", C.c_void_p),
                ("snp", C.c_void_p), ("allele", C.c_void_p), ("qual", C.c_void_p),
                ("is_porec", C.c_void_p), ("on_device", C.c_int32)]


class QhGraphOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("weight_mode", C.c_int32), ("linkage_k", C.c_int32),
                ("dense", C.c_int32), ("storage", C.c_int32), ("porec_alpha", C.c_double)]


class QhBsbOpts(C.Structure):
    _fields_ = [("replicas", C.c_int32), ("steps", C.c_int32), ("schedule", C.c_int32),
                ("precision", C.c_int32), ("dt", C.c_double), ("a0", C.c_double),
                ("c0", C.c_double), ("seed", C.c_uint64), ("replica_base", C.c_int32),
                ("check_every", C.c_int32), ("patience", C.c_int32), ("refine_max", C.c_int32),
                ("step_kernel", C.c_int32), ("sb_variant", C.c_int32),
                ("deform_h", C.c_double), ("deform_tries", C.c_int32), ("check_mode", C.c_int32),
                ("track_best", C.c_int32)]

class QhRefineState(C.Structure):
    _fields_ = [("iterations_done", C.c_int32), ("flips", C.c_void_p), ("gauge", C.c_void_p),
                ("refining", C.c_void_p), ("solves", C.c_void_p), ("deform", C.c_void_p),
                ("tries", C.c_void_p)]


# simulated-bifurcation variants (QH_SB_*)
SB_VARIANTS = {"ballistic": 0, "discrete": 1, "adiabatic": 2}


def _sb(variant):
    return SB_VARIANTS[variant] if isinstance(variant, str) else int(variant)
STEP_KERNELS = ["cta-bn128-s3", "cta-bn128-s2-x3", "cta-bn64-s2-x4", "cta-bn256-s2-x2",
                "persistent-bn128", "persistent-bn64-tma-state",
                "multistep-jres-group", "multistep-stream-tile", "multistep-jres-tile",
                "multistep-stream-group",
                # CSR storage (FP32 or BF16): 4 or 8 replicas per lane
                "csr-lane4", "csr-lane8",
                # CSR storage, BF16: the band on the tensor cores + the lane-8 remainder step
                "csr-band8"]


class QhError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "QH_OK", 1: "QH_EINVAL", 2: "QH_ENOMEM", 3: "QH_ECUDA", 4: "QH_ETIMEOUT",
           5: "QH_EUNSUPPORTED"}

P, PP = C.c_void_p, C.POINTER(C.c_void_p)
I32, I64, D = C.c_int32, C.c_int64, C.c_double
_SIGS = {
    "qh_create": (C.c_int, [PP, C.c_int, P]),
    "qh_destroy": (None, [P]),
    "qh_status_str": (C.c_char_p, [C.c_int]),
    "qh_last_error": (C.c_char_p, [P]),
    "qh_build_graph": (C.c_int, [P, C.POINTER(QhFragments), C.POINTER(QhGraphOpts), PP]),
    "qh_graph_info": (C.c_int, [P, P, P, P, I32, P, P]),
    "qh_graph_edges": (C.c_int, [P, P, P, P, P]),
    "qh_graph_blocks": (C.c_int, [P, P, P, P]),
    "qh_graph_free": (None, [P]),
    "qh_bsb_solve": (C.c_int, [P, P, C.POINTER(QhBsbOpts), PP]),
    "qh_bsb_solve_blocks": (C.c_int, [P, P, C.POINTER(QhBsbOpts), P, I32, PP]),
    "qh_bsb_solve_resume": (C.c_int, [P, P, C.POINTER(QhBsbOpts), C.POINTER(QhRefineState), PP]),
    "qh_solution_refine_state": (C.c_int, [P, C.POINTER(QhRefineState)]),
    "qh_solution_check_trace": (C.c_int, [P, P, P, P]),
    "qh_solution_set_block": (C.c_int, [P, P, I32, P, D, I32, I32, I32]),
    "qh_solution_block": (C.c_int, [P, P, I32, P, P, P, P, P]),
    "qh_solution_spins": (C.c_int, [P, P, P]),
    "qh_solution_cuts": (C.c_int, [P, P, P]),
    "qh_solution_timing": (C.c_int, [P, P, P, P, P]),
    "qh_solution_free": (None, [P]),
    "qh_phase": (C.c_int, [P, P, P, P, P, P, I32]),
    "qh_debug_matvec": (C.c_int, [P, P, I32, I32, P, P]),
    "qh_debug_steps": (C.c_int, [P, P, I32, I32, P, P, I32, I32, I32, D, D, P]),
    "qh_debug_wait_timeout": (C.c_int, [P, I32]),
    "qh_debug_fail_alloc": (C.c_int, [P, I64]),
    "qh_debug_steps_v": (C.c_int, [P, P, I32, I32, P, P, I32, I32, I32, D, D, P, I32, I32, P]),
    "qh_debug_layout": (C.c_int, [P, P, P, P, P]),
    "qh_debug_init_state": (C.c_int, [P, P, I32, I32, C.c_uint64, I32, P, P]),
    "qh_debug_run_trace": (C.c_int, [P, P, I32, I32, I32, I32, I32, P, P, P]),
    "qh_matvec_bf16_noalloc": (C.c_int, [P, P, I32, P, P]),
    "qh_solution_kernel": (C.c_char_p, [P]),
    "qh_tuning_report": (C.c_char_p, [P]),
    "qh_kernel_launches": (C.c_int64, []),
}

_lib = None


def lib():
    """Load libqhap.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libqhap.so not found at {LIB_PATH}; run "
                          "paper_2603_25762_gb300.build.build() first (no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def __getattr__(name):
    if name in _SIGS:
        return getattr(lib(), name)
    raise AttributeError(name)


def kernel_launches():
    """CUDA kernels libqhap has launched in this process."""
    return int(lib().qh_kernel_launches())


def _ptr(a):
    """Host numpy array or device torch tensor -> raw address (None stays NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Graph:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.h = handle
        n, nb, nnz, nt = I32(), I32(), I64(), I64()
        lib().qh_graph_info(handle, C.byref(n), C.byref(nb), None, 0, C.byref(nnz), C.byref(nt))
        self.n_nodes, self.n_blocks, self.nnz, self.n_tiles = n.value, nb.value, nnz.value, nt.value

    def block_sizes(self):
        out = np.zeros(max(self.n_blocks, 1), np.int32)
        lib().qh_graph_info(self.h, None, None, _ptr(out), self.n_blocks, None, None)
        return out[: self.n_blocks]

    def edges(self):
        rp = np.zeros(self.n_nodes + 1, np.int64)
        col = np.zeros(max(self.nnz, 1), np.int32)
        w = np.zeros(max(self.nnz, 1), np.float64)
        self.ctx._check(lib().qh_graph_edges(self.ctx.h, self.h, _ptr(rp), _ptr(col), _ptr(w)))
        return rp, col[: self.nnz], w[: self.nnz]

    def blocks(self):
        bo = np.zeros(max(self.n_nodes, 1), np.int32)
        lo = np.zeros(max(self.n_nodes, 1), np.int32)
        self.ctx._check(lib().qh_graph_blocks(self.ctx.h, self.h, _ptr(bo), _ptr(lo)))
        return bo[: self.n_nodes], lo[: self.n_nodes]

    def layout(self):
        n_pad = I32()
        pidx = np.zeros(max(self.n_nodes, 1), np.int32)
        c0 = np.zeros(max(self.n_blocks, 1), np.float64)
        self.ctx._check(lib().qh_debug_layout(self.ctx.h, self.h, C.byref(n_pad), _ptr(pidx),
                                              _ptr(c0)))
        return n_pad.value, pidx[: self.n_nodes], c0[: self.n_blocks]

    def free(self):
        if self.h:
            lib().qh_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _refine_struct(done, st):
    return QhRefineState(int(done), _ptr(st["flips"]), _ptr(st["gauge"]), _ptr(st["refining"]),
                         _ptr(st["solves"]), _ptr(st["deform"]), _ptr(st["tries"]))


class Solution:
    def __init__(self, ctx, handle, n_blocks, R):
        self.ctx, self.h, self.n_blocks, self.R = ctx, handle, n_blocks, R

    def block(self, b, size=None):
        cut, br, sr, it = D(), I32(), I32(), I32()
        sp = np.zeros(max(size or 0, 1), np.int8)
        self.ctx._check(lib().qh_solution_block(self.ctx.h, self.h, b, _ptr(sp) if size else None,
                                                C.byref(cut), C.byref(br), C.byref(sr),
                                                C.byref(it)))
        return {"best_cut": cut.value, "best_replica": br.value, "steps_run": sr.value,
                "iterations": it.value, "spins": sp[:size] if size else None}

    def set_block(self, b, spins, best_cut, best_replica, steps_run, iterations):
        """Import block b's result (as block() returns it in another process)."""
        sp = _np(spins, np.int8)
        self.ctx._check(lib().qh_solution_set_block(self.ctx.h, self.h, b, _ptr(sp),
                                                    float(best_cut), int(best_replica),
                                                    int(steps_run), int(iterations)))

    def refine_state(self, n_nodes):
        """The SNP refinement's state after this solve (qh_solution_refine_state), as a
        dict of host arrays that Context.solve(resume=...) continues from."""
        n = max(n_nodes, 1)
        nb = max(self.n_blocks, 1)
        st = {"flips": np.zeros(n, np.int32), "gauge": np.zeros(n, np.int8),
              "refining": np.zeros(nb, np.int32), "solves": np.zeros(nb, np.int32),
              "deform": np.zeros(nb, np.float32), "tries": np.zeros(nb, np.int32)}
        rs = _refine_struct(0, st)
        r = lib().qh_solution_refine_state(self.h, C.byref(rs))
        if r != QH_OK:
            raise QhError(r, "no refinement state (READ mode, or blocks imported)")
        out = {k: (v[:n_nodes] if k in ("flips", "gauge") else v[: self.n_blocks])
               for k, v in st.items()}
        out["iterations_done"] = rs.iterations_done
        return out

    def check_trace(self):
        """The first solve's energy checks: (check_every, array [checks][n_blocks] of each
        block's best cut per check, NaN where the block was not running)."""
        n, ce = I32(), I32()
        self.ctx._check(lib().qh_solution_check_trace(self.h, C.byref(n), C.byref(ce), None))
        tr = np.zeros(max(n.value * self.n_blocks, 1))
        self.ctx._check(lib().qh_solution_check_trace(self.h, C.byref(n), None, _ptr(tr)))
        return ce.value, tr[: n.value * self.n_blocks].reshape(n.value, self.n_blocks)

    def spins(self, n_nodes):
        s = np.zeros(max(n_nodes, 1), np.int8)
        self.ctx._check(lib().qh_solution_spins(self.ctx.h, self.h, _ptr(s)))
        return s[:n_nodes]

    def cuts(self):
        c = np.zeros(max(self.n_blocks * self.R, 1))
        self.ctx._check(lib().qh_solution_cuts(self.ctx.h, self.h, _ptr(c)))
        return c[: self.n_blocks * self.R].reshape(self.n_blocks, self.R)

    def timing(self):
        a, b, n, su = D(), D(), I64(), D()
        lib().qh_solution_timing(self.h, C.byref(a), C.byref(b), C.byref(n), C.byref(su))
        return {"kernel": lib().qh_solution_kernel(self.h).decode(),
                "solve_ms": a.value, "step_ms": b.value, "n_step_launches": n.value,
                "spin_updates": su.value}

    def free(self):
        if self.h:
            lib().qh_solution_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """One library context on one CUDA device (optionally on a caller's stream)."""

    def __init__(self, device=0, stream=None):
        h = C.c_void_p()
        st = lib().qh_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
        if st != QH_OK:
            raise QhError(st, "qh_create failed")
        self.h = h

    def _check(self, st):
        if st != QH_OK:
            raise QhError(st, lib().qh_last_error(self.h).decode())

    def build_graph(self, fr=None, mode=MODE_READ, weight_mode=WEIGHT_SIGNED, linkage_k=10,
                    dense=False, porec_alpha=0.1, arrays=None, on_device=False,
                    storage=STORAGE_AUTO):
        """fr: a synth.Fragments (host); or arrays=(n_snps, frag_ptr, snp, allele, qual, is_porec)
        as numpy (host) or torch CUDA tensors with on_device=True."""
        if arrays is None:
            arrays = (fr.n_snps, _np(fr.frag_ptr, np.int64), _np(fr.snp, np.int32),
                      _np(fr.allele, np.int8), _np(fr.qual, np.uint8), _np(fr.is_porec, np.uint8))
        n_snps, fp, snp, al, q, pc = arrays
        f = QhFragments(int(fp.shape[0]) - 1, int(n_snps), _ptr(fp), _ptr(snp), _ptr(al), _ptr(q),
                        _ptr(pc), 1 if on_device else 0)
        o = QhGraphOpts(mode, weight_mode, linkage_k, 1 if dense else 0, storage, porec_alpha)
        g = C.c_void_p()
        self._check(lib().qh_build_graph(self.h, C.byref(f), C.byref(o), C.byref(g)))
        return Graph(self, g)

    def solve(self, g, replicas=32, steps=1000, precision=PREC_FP32, seed=1, dt=1.0, a0=1.0,
              c0=0.0, schedule=SCHED_LINEAR, replica_base=0, check_every=0, patience=0,
              refine_max=15, step_kernel=None, variant="ballistic", deform_h=0.0,
              deform_tries=0, blocks=None, check_mode=0, track_best=False, resume=None):
        """step_kernel: None = the default (autotuned on BF16 tile storage), or a name
        from STEP_KERNELS: the tile variants for BF16 tile storage, "csr-lane4" /
        "csr-lane8" for CSR storage.
        variant: "ballistic" (bSB), "discrete" (dSB) or "adiabatic" (aSB), or the
        QH_SB_* value itself.
        deform_h, deform_tries: the SNP refinement's adaptive deformation (0 = off): up
        to deform_tries re-solves of a block whose cut is <= 0, with a field along the
        incumbent of strength deform_h 2^(k-1).
        blocks: None = every block; else the block indices to solve (the others stay
        unsolved, see qh_bsb_solve_blocks).
        check_mode: where early-stop checks run, 0 = inside the multi-step launch when it
        applies, 1 = between launches (qh_bsb_opts.check_mode).
        track_best: report the best result reached at any check (every check_every
        steps) or at the end, instead of the final state's.
        resume: a SNP refinement state (Solution.refine_state()) to continue from, up to
        refine_max solves in all (qh_bsb_solve_resume)."""
        sk = -1 if step_kernel is None else STEP_KERNELS.index(step_kernel)
        o = QhBsbOpts(replicas, steps, schedule, precision, dt, a0, c0, seed, replica_base,
                      check_every, patience, refine_max, sk, _sb(variant), deform_h,
                      deform_tries, check_mode, 1 if track_best else 0)
        s = C.c_void_p()
        if resume is not None:
            st = {"flips": _np(resume["flips"], np.int32), "gauge": _np(resume["gauge"], np.int8),
                  "refining": _np(resume["refining"], np.int32),
                  "solves": _np(resume["solves"], np.int32),
                  "deform": _np(resume["deform"], np.float32),
                  "tries": _np(resume["tries"], np.int32)}
            rs = _refine_struct(resume["iterations_done"], st)
            self._check(lib().qh_bsb_solve_resume(self.h, g.h, C.byref(o), C.byref(rs),
                                                  C.byref(s)))
        elif blocks is None:
            self._check(lib().qh_bsb_solve(self.h, g.h, C.byref(o), C.byref(s)))
        else:
            sel = _np(blocks, np.int32)
            self._check(lib().qh_bsb_solve_blocks(self.h, g.h, C.byref(o),
                                                  _ptr(sel) if sel.size else None,
                                                  int(sel.size), C.byref(s)))
        return Solution(self, s, g.n_blocks, replicas)

    def phase(self, g, sol, n_snps, out=None):
        """Host outputs by default; pass out=(hap1, hap2, block_id) torch CUDA tensors to keep
        them on the device."""
        if out is None:
            hap1 = np.zeros(max(n_snps, 1), np.int8)
            hap2 = np.zeros(max(n_snps, 1), np.int8)
            bid = np.zeros(max(n_snps, 1), np.int32)
            self._check(lib().qh_phase(self.h, g.h, sol.h, _ptr(hap1), _ptr(hap2), _ptr(bid), 0))
            return hap1[:n_snps], hap2[:n_snps], bid[:n_snps]
        hap1, hap2, bid = out
        self._check(lib().qh_phase(self.h, g.h, sol.h, _ptr(hap1), _ptr(hap2), _ptr(bid), 1))
        return hap1, hap2, bid

    def debug_matvec(self, g, precision, R, x, z):
        self._check(lib().qh_debug_matvec(self.h, g.h, precision, R, _ptr(x), _ptr(z)))

    def debug_steps(self, g, precision, R, x, y, t0, nsteps, steps, dt=1.0, a0=1.0, c0=None,
                    step_kernel=None, variant="ballistic", field=None):
        """step_kernel: None = default kernel, or a name from STEP_KERNELS.
        field: per-block deformation field strengths (None = no field)."""
        c0a = None if c0 is None else _np(c0, np.float64)
        fa = None if field is None else _np(field, np.float64)
        sk = -1 if step_kernel is None else STEP_KERNELS.index(step_kernel)
        self._check(lib().qh_debug_steps_v(self.h, g.h, precision, R, _ptr(x), _ptr(y), t0,
                                           nsteps, steps, dt, a0,
                                           _ptr(c0a) if c0a is not None else None, sk,
                                           _sb(variant),
                                           _ptr(fa) if fa is not None else None))

    def debug_init_state(self, g, R, x, y, replica_base=0, seed=1, it=0):
        """The solver's initial x, y (torch CUDA float32 tensors [R][n_pad]) for replicas
        replica_base .. replica_base + R - 1 of refinement iteration `it`."""
        self._check(lib().qh_debug_init_state(self.h, g.h, R, replica_base, seed, it, _ptr(x),
                                              _ptr(y)))

    def debug_run_trace(self, g, R, step_kernel, steps, u0, nu):
        """Step timeline of one multi-step launch: (stamps uint64[n_ctas, nu, 4, 32],
        items int32[n_ctas, 4]); see qh_debug_run_trace for the events."""
        sk = STEP_KERNELS.index(step_kernel) if isinstance(step_kernel, str) else step_kernel
        n = I32()
        self._check(lib().qh_debug_run_trace(self.h, g.h, R, sk, steps, u0, nu, None, None,
                                             C.byref(n)))
        stamps = np.zeros((n.value, nu, 4, 32), np.uint64)
        items = np.zeros((n.value, 4), np.int32)
        self._check(lib().qh_debug_run_trace(self.h, g.h, R, sk, steps, u0, nu, _ptr(stamps),
                                             _ptr(items), C.byref(n)))
        return stamps, items

    def debug_wait_timeout(self, which=0):
        """Failure-detection hook: a bounded device wait that expires (raises QhError
        with status QH_ETIMEOUT after about a second)."""
        self._check(lib().qh_debug_wait_timeout(self.h, which))

    def debug_fail_alloc(self, after):
        """Error-path hook: the next `after` device allocations succeed, later ones fail
        with QH_ENOMEM; after = -1 turns it off."""
        self._check(lib().qh_debug_fail_alloc(self.h, after))

    def matvec_bf16_noalloc(self, g, R, x, z):
        """J x X in BF16 without any device allocation (fixed 8.5 MiB library array)."""
        self._check(lib().qh_matvec_bf16_noalloc(self.h, g.h, R, _ptr(x), _ptr(z)))

    def tuning_report(self):
        return lib().qh_tuning_report(self.h).decode()

    def close(self):
        if self.h:
            lib().qh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
