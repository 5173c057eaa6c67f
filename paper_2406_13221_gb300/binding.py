"""Thin ctypes binding of libhelr.so (declared in include/he_lr.h).

Argument marshalling only: every computation runs in the CUDA library.  The
module raises ImportError-free but loud errors: ``load()`` fails if the
library has not been built, and every call that returns a non-zero status
raises ``HeError`` with the library's message.  There is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhelr.so")

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ELEVEL, HE_ESCALE, HE_ECUDA, HE_ETIMEOUT, HE_EINTERNAL, HE_EKEY = range(9)
CODES = {1: "HE_EINVAL", 2: "HE_ENOMEM", 3: "HE_ELEVEL", 4: "HE_ESCALE", 5: "HE_ECUDA",
         6: "HE_ETIMEOUT", 7: "HE_EINTERNAL", 8: "HE_EKEY"}
FULL_BATCH, MINI_BATCH = 0, 1
FIRST_ORDER = 0x100  # OR into the mode: the first-order NAG baseline (no Bbar)
G8, G16 = 0, 1


class HeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (CODES.get(code, code), msg))
        self.code = code


class he_params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int), ("n_q", ctypes.c_int), ("q0_bits", ctypes.c_int),
                ("qi_bits", ctypes.c_int), ("p_bits", ctypes.c_int), ("sigma", ctypes.c_double),
                ("bits", ctypes.POINTER(ctypes.c_int)), ("secret_hw", ctypes.c_int)]


class he_boot_params(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("K", ctypes.c_int), ("double_angles", ctypes.c_int),
                ("degree", ctypes.c_int), ("scale_out", ctypes.c_double), ("level_out", ctypes.c_int)]


class he_lr_sched(ctypes.Structure):
    _fields_ = [("max", ctypes.c_double), ("min", ctypes.c_double), ("T", ctypes.c_double),
                ("power", ctypes.c_double)]


class he_lr_stats(ctypes.Structure):
    _fields_ = [("sec_setup", ctypes.c_double), ("sec_iter_avg", ctypes.c_double),
                ("sec_update_avg", ctypes.c_double), ("keyswitches", ctypes.c_uint64),
                ("n_blocks", ctypes.c_int), ("g", ctypes.c_int), ("m", ctypes.c_int),
                ("max_abs_ip", ctypes.c_double)]


# every exported symbol of include/he_lr.h with (restype, argtypes)
_vp, _i, _u64, _i64, _d, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64,
                                ctypes.c_double, ctypes.c_size_t)
_pp = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "he_ctx_create": (_i, [ctypes.POINTER(he_params), _vp, _pp]),
    "he_ctx_destroy": (_i, [_vp]),
    "he_last_error": (ctypes.c_char_p, [_vp]),
    "he_ctx_primes": (_i, [_vp, _vp, _sz]),
    "he_gauss_table": (_i, [_d, _vp, _sz, ctypes.POINTER(ctypes.c_size_t)]),
    "he_zeta_table": (_i, [_i, _vp, _vp]),
    "he_keygen": (_i, [_vp, _u64, _vp, _sz]),
    "he_encode": (_i, [_vp, _vp, _vp, _sz, _i, _d, _pp]),
    "he_decode": (_i, [_vp, _vp, _vp, _vp, _sz]),
    "he_encrypt": (_i, [_vp, _vp, _u64, _pp]),
    "he_decrypt": (_i, [_vp, _vp, _pp]),
    "he_ct_export": (_i, [_vp, _vp, _sz, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "he_ct_import": (_i, [_vp, _vp, _sz, _i, _d, _pp]),
    "he_pt_export": (_i, [_vp, _vp, _sz, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "he_ct_level": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "he_ct_free": (_i, [_vp]),
    "he_pt_free": (_i, [_vp]),
    "he_add": (_i, [_vp, _vp, _vp, _pp]),
    "he_sub": (_i, [_vp, _vp, _vp, _pp]),
    "he_mul": (_i, [_vp, _vp, _vp, _pp]),
    "he_rescale": (_i, [_vp, _vp, _pp]),
    "he_moddrop": (_i, [_vp, _vp, _i, _pp]),
    "he_rotate": (_i, [_vp, _vp, _i64, _pp]),
    "he_cmul": (_i, [_vp, _vp, _d, _d, _pp]),
    "he_cadd": (_i, [_vp, _vp, _d, _pp]),
    "he_ptmul": (_i, [_vp, _vp, _vp, _pp]),
    "he_set_scale": (_i, [_vp, _d]),
    "he_ntt_forward": (_i, [_vp, _vp, _sz, _vp, _i]),
    "he_ntt_inverse": (_i, [_vp, _vp, _sz, _vp, _i]),
    "he_keyswitch_batch": (_i, [_vp, _vp, _vp, _i, _i, _u64]),
    "he_autotune": (_i, [_vp, ctypes.c_char_p, _i, ctypes.POINTER(_i)]),
    "he_ks_wave": (_i, [_vp, _i]),
    "he_galois_elt": (_u64, [_vp, _i64]),
    "he_lr_job_create": (_i, [_vp, _vp, _vp, _sz, _sz, _i, _sz, _i, _d, _u64, _u64, _i, _pp]),
    "he_lr_job_step": (_i, [_vp, _i, he_lr_sched]),
    "he_lr_job_weights": (_i, [_vp, _i, _vp, _sz]),
    "he_lr_job_state": (_i, [_vp, _pp, _pp]),
    "he_lr_job_block_grad": (_i, [_vp, _i, _pp]),
    "he_lr_job_input": (_i, [_vp, _i, _i, _pp]),
    "he_lr_job_info": (_i, [_vp, ctypes.POINTER(he_lr_stats)]),
    "he_lr_job_step_io": (_i, [_vp, _i, he_lr_sched, _vp, _vp]),
    "he_launch_count": (_u64, []),
    "he_rescale_noalloc": (_i, [_vp, _vp, _vp, _i, _i]),
    "he_lr_job_set_batch": (_i, [_vp, _i]),
    "he_lr_job_set_graph": (_i, [_vp, _i]),
    "he_prof_enable": (_i, [_vp, _i]),
    "he_prof_read": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_d), ctypes.POINTER(_u64)]),
    "he_prof_read2": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "he_prof_keyswitches": (_i, [_vp, _vp, _sz]),
    "he_set_rotation_radix": (_i, [_vp, _i]),
    "he_keygen_galois": (_i, [_vp, _vp, _sz]),
    "he_lr_job_set_refresh": (_i, [_vp, ctypes.POINTER(he_boot_params)]),
    "he_boot_keys": (_i, [_vp, ctypes.POINTER(he_boot_params), _vp, _sz, ctypes.POINTER(_sz)]),
    "he_bootstrap": (_i, [_vp, _vp, ctypes.POINTER(he_boot_params), _pp]),
    "he_bootstrap_batch": (_i, [_vp, _vp, _i, _vp, _i, ctypes.POINTER(he_boot_params)]),
    "he_rotsum": (_i, [_vp, _vp, _vp, _sz, _pp]),
    "he_rotsum_batch": (_i, [_vp, _vp, _vp, _i, _i, _vp, _sz]),
    "he_mul_relin_batch": (_i, [_vp, _vp, _vp, _vp, _i, _i]),
    "he_rescale_batch": (_i, [_vp, _vp, _vp, _i, _i]),
    "he_rotate_batch": (_i, [_vp, _vp, _vp, _i, _i, ctypes.c_int64]),
    "he_ks_tile": (_i, [_vp, _i]),
    "he_set_ks_tile": (_i, [_vp, _i]),
    "he_set_hoist_form": (_i, [_vp, _i]),
    "he_hoist_form": (_i, [_vp, _i]),
    "he_hoist_tensor_launches": (ctypes.c_ulonglong, [_vp]),
    "he_check_device": (_i, [_vp]),
    "he_selftest_bounded_wait": (_i, [_vp, _i]),
    "he_lr_job_free": (_i, [_vp]),
    "he_lr_multi_create": (_i, [_vp, _vp, _sz, _i, _pp]),
    "he_lr_multi_step": (_i, [_vp, _i, he_lr_sched]),
    "he_lr_multi_free": (_i, [_vp]),
    "he_lr_train": (_i, [_vp, _vp, _vp, _sz, _sz, _i, he_lr_sched, _i, _sz, _i, _u64, _u64, _vp, _sz,
                         ctypes.POINTER(he_lr_stats)]),
    "he_lr_iteration": (_i, [_vp, _vp, _sz, _vp, _vp, _vp, _i, _i, _d, _d, _d, _vp, _pp, _pp]),
    "he_refresh": (_i, [_vp, _vp, _i, _d, _u64, _pp]),
    "he_lr_bbar": (_i, [_vp, _vp, _sz, _sz, _sz, _sz, _sz, _vp]),
    "he_lr_bbar_batches": (_i, [_vp, _vp, _vp, _sz, _sz, _sz, _sz, _vp]),
}

_lib = None


def load():
    """Load the built library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError("libhelr.so is not built (%s); run paper_2406_13221_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Context:
    """One he_ctx: parameter set, tables, keys; kernels run on `stream`."""

    def __init__(self, log_n=13, n_q=9, q0_bits=60, qi_bits=40, p_bits=60, sigma=3.2, stream=None, bits=None,
                 secret_weight=0):
        self.L = load()
        barr = None
        if bits is not None:
            if len(bits) != n_q:
                raise ValueError("one bit width per ciphertext prime")
            barr = (ctypes.c_int * n_q)(*bits)
        p = he_params(log_n, n_q, q0_bits, qi_bits, p_bits, sigma, barr, int(secret_weight))
        h = ctypes.c_void_p()
        rc = self.L.he_ctx_create(ctypes.byref(p), stream, ctypes.byref(h))
        if rc:
            raise HeError(rc, "he_ctx_create failed")
        self.h = h
        self.log_n, self.n, self.nslots, self.n_q = log_n, 1 << log_n, 1 << (log_n - 1), n_q
        pr = np.zeros(n_q + 1, np.uint64)
        self.check(self.L.he_ctx_primes(self.h, _ptr(pr), n_q + 1))
        self.primes = [int(x) for x in pr]

    def check(self, rc):
        if rc:
            raise HeError(rc, self.L.he_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.he_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def out(self):
        return ctypes.c_void_p()

    # keys / encoding
    def keygen(self, seed, rotations=()):
        r = np.asarray(list(rotations), np.int64)
        self.check(self.L.he_keygen(self.h, seed, _ptr(r) if len(r) else None, len(r)))

    def keygen_galois(self, gals):
        g = np.asarray(gals, np.uint64)
        self.check(self.L.he_keygen_galois(self.h, _ptr(g), len(g)))

    def boot_keys(self, slots, K, r, deg, scale_out, level_out):
        """rotation amounts a bootstrap needs"""
        p = he_boot_params(slots, K, r, deg, scale_out, level_out)
        n = ctypes.c_size_t()
        self.check(self.L.he_boot_keys(self.h, ctypes.byref(p), None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, np.int64)
        self.check(self.L.he_boot_keys(self.h, ctypes.byref(p), _ptr(out), n.value, ctypes.byref(n)))
        return [int(x) for x in out]

    def bootstrap(self, ct, slots, K, r, deg, scale_out, level_out):
        p = he_boot_params(slots, K, r, deg, scale_out, level_out)
        o = ctypes.c_void_p()
        self.check(self.L.he_bootstrap(self.h, ct.h, ctypes.byref(p), ctypes.byref(o)))
        return Ct(self, o)

    def bootstrap_batch(self, din, in_level, dout, batch, slots, K, r, deg, scale_out, level_out):
        p = he_boot_params(slots, K, r, deg, scale_out, level_out)
        self.check(self.L.he_bootstrap_batch(self.h, din, in_level, dout, batch, ctypes.byref(p)))

    def galois_elt(self, r):
        return int(self.L.he_galois_elt(self.h, int(r)))

    def encode(self, z, level, scale):
        z = np.asarray(z, np.complex128)
        re, im = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        o = self.out()
        self.check(self.L.he_encode(self.h, _ptr(re), _ptr(im), len(z), level, float(scale), ctypes.byref(o)))
        return Pt(self, o)

    def decode(self, pt):
        re = np.zeros(self.nslots)
        im = np.zeros(self.nslots)
        self.check(self.L.he_decode(self.h, pt.h, _ptr(re), _ptr(im), self.nslots))
        return re + 1j * im

    def encrypt(self, pt, seed):
        o = self.out()
        self.check(self.L.he_encrypt(self.h, pt.h, seed, ctypes.byref(o)))
        return Ct(self, o)

    def decrypt(self, ct):
        o = self.out()
        self.check(self.L.he_decrypt(self.h, ct.h, ctypes.byref(o)))
        return Pt(self, o)

    def import_ct(self, words, level, scale):
        w = np.ascontiguousarray(words, np.uint64)
        o = self.out()
        self.check(self.L.he_ct_import(self.h, _ptr(w), w.size, level, float(scale), ctypes.byref(o)))
        return Ct(self, o)

    # operations
    def _op(self, name, *args):
        o = self.out()
        self.check(getattr(self.L, name)(self.h, *args, ctypes.byref(o)))
        return Ct(self, o)

    def add(self, a, b):
        return self._op("he_add", a.h, b.h)

    def sub(self, a, b):
        return self._op("he_sub", a.h, b.h)

    def mul(self, a, b):
        return self._op("he_mul", a.h, b.h)

    def rescale(self, a):
        return self._op("he_rescale", a.h)

    def moddrop(self, a, level):
        return self._op("he_moddrop", a.h, level)

    def rotate(self, a, r):
        return self._op("he_rotate", a.h, int(r))

    def rotsum(self, a, rots):
        r = np.asarray(rots, np.int64)
        o = ctypes.c_void_p()
        self.check(self.L.he_rotsum(self.h, a.h, _ptr(r), len(r), ctypes.byref(o)))
        return Ct(self, o)

    def cmul(self, a, c, const_scale):
        return self._op("he_cmul", a.h, float(c), float(const_scale))

    def cadd(self, a, c):
        return self._op("he_cadd", a.h, float(c))

    def ptmul(self, a, pt):
        return self._op("he_ptmul", a.h, pt.h)

    def refresh(self, ct, level, scale, seed):
        return self._op("he_refresh", ct.h, int(level), float(scale), seed)

    # device-pointer primitives
    def ntt_forward(self, dptr, nlimbs, prime_of):
        p = np.asarray(prime_of, np.int32)
        self.check(self.L.he_ntt_forward(self.h, dptr, nlimbs, _ptr(p), len(p)))

    def ntt_inverse(self, dptr, nlimbs, prime_of):
        p = np.asarray(prime_of, np.int32)
        self.check(self.L.he_ntt_inverse(self.h, dptr, nlimbs, _ptr(p), len(p)))

    def prof_enable(self, on=True):
        self.check(self.L.he_prof_enable(self.h, int(on)))

    def prof_read(self, cls):
        """(milliseconds, work units, launches, second work count, DRAM limbs) of a timing class."""
        ms, units, n, u2, u3 = (ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64(), ctypes.c_double(),
                                ctypes.c_double())
        self.check(self.L.he_prof_read(self.h, cls, ctypes.byref(ms), ctypes.byref(units), ctypes.byref(n)))
        self.check(self.L.he_prof_read2(self.h, cls, ctypes.byref(u2), ctypes.byref(u3)))
        return ms.value, units.value, n.value, u2.value, u3.value

    def set_rotation_radix(self, log2_radix):
        """Rotate-and-sum steps as hoisted groups of 2^log2_radix positions."""
        self.check(self.L.he_set_rotation_radix(self.h, int(log2_radix)))

    def prof_keyswitches(self):
        """Key switches issued since profiling was enabled, per input limb count."""
        out = np.zeros(64)
        self.check(self.L.he_prof_keyswitches(self.h, _ptr(out), len(out)))
        return {nl: int(v) for nl, v in enumerate(out) if v}

    def rescale_noalloc(self, din, dout, batch, level):
        self.check(self.L.he_rescale_noalloc(self.h, din, dout, batch, level))

    def autotune(self, path=None, items=0):
        """Choose the key-switch wave per level (he_autotune); returns the number of levels measured."""
        n = ctypes.c_int()
        self.check(self.L.he_autotune(self.h, None if path is None else os.fsencode(path), int(items), ctypes.byref(n)))
        return n.value

    def ks_tile(self, level):
        v = self.L.he_ks_tile(self.h, level)
        if v < 0:
            raise HeError(-v, "he_ks_tile")
        return v

    def set_ks_tile(self, tile):
        self.check(self.L.he_set_ks_tile(self.h, int(tile)))

    def set_hoist_form(self, form):
        """0: hoisted inner products on the CUDA cores; 1: on the tensor cores where they
        apply; -1: the form he_autotune chose per limb count."""
        self.check(self.L.he_set_hoist_form(self.h, int(form)))

    def hoist_form(self, level):
        v = self.L.he_hoist_form(self.h, int(level))
        if v < 0:
            raise HeError(-v, "he_hoist_form")
        return v

    def hoist_tensor_launches(self):
        return int(self.L.he_hoist_tensor_launches(self.h))

    def check_device(self):
        """Raise HeError(HE_ETIMEOUT) if a bounded device-side wait expired."""
        self.check(self.L.he_check_device(self.h))

    def selftest_bounded_wait(self, arrive):
        self.check(self.L.he_selftest_bounded_wait(self.h, int(arrive)))

    def ks_wave(self, level):
        w = self.L.he_ks_wave(self.h, int(level))
        if w <= 0:
            self.check(-w)
        return w

    def rotsum_batch(self, din, dout, batch, level, rots):
        r = np.asarray(rots, np.int64)
        self.check(self.L.he_rotsum_batch(self.h, din, dout, batch, level, _ptr(r), len(r)))

    def keyswitch_batch(self, din, dout, batch, level, gal):
        self.check(self.L.he_keyswitch_batch(self.h, din, dout, batch, level, gal))

    def mul_relin_batch(self, da, db, dout, batch, level):
        self.check(self.L.he_mul_relin_batch(self.h, da, db, dout, batch, level))

    def rescale_batch(self, din, dout, batch, level):
        self.check(self.L.he_rescale_batch(self.h, din, dout, batch, level))

    def rotate_batch(self, din, dout, batch, level, r):
        self.check(self.L.he_rotate_batch(self.h, din, dout, batch, level, int(r)))


class Ct:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def info(self):
        lv, sc = ctypes.c_int(), ctypes.c_double()
        self.ctx.check(self.ctx.L.he_ct_level(self.h, ctypes.byref(lv), ctypes.byref(sc)))
        return lv.value, sc.value

    @property
    def level(self):
        return self.info()[0]

    @property
    def scale(self):
        return self.info()[1]

    def set_scale(self, s):
        self.ctx.check(self.ctx.L.he_set_scale(self.h, float(s)))

    def export(self):
        lv, sc = self.info()
        w = np.zeros((2, lv + 1, self.ctx.n), np.uint64)
        self.ctx.check(self.ctx.L.he_ct_export(self.h, _ptr(w), w.size, None, None))
        return w

    def __del__(self):
        try:
            if self.h:
                self.ctx.L.he_ct_free(self.h)
                self.h = None
        except Exception:
            pass


class Pt:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def export(self):
        lv, sc = ctypes.c_int(), ctypes.c_double()
        w = np.zeros((self.ctx.n_q, self.ctx.n), np.uint64)
        self.ctx.check(self.ctx.L.he_pt_export(self.h, _ptr(w), w.size, ctypes.byref(lv), ctypes.byref(sc)))
        return w[:lv.value + 1].copy(), lv.value, sc.value

    def __del__(self):
        try:
            if self.h:
                self.ctx.L.he_pt_free(self.h)
                self.h = None
        except Exception:
            pass


class Job:
    """he_lr_job: client precompute + encryption at creation, one iteration per step()."""

    def __init__(self, ctx, X, y, mode=FULL_BATCH, batch_rows=1024, poly=G8, log_scale=40.0,
                 enc_seed=3, key_seed=2, batch_blocks=0):
        self.ctx = ctx
        X = np.ascontiguousarray(X, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        n, f = X.shape
        h = ctypes.c_void_p()
        ctx.check(ctx.L.he_lr_job_create(ctx.h, _ptr(X), _ptr(y), n, f, mode, batch_rows, poly, log_scale,
                                         enc_seed, key_seed, batch_blocks, ctypes.byref(h)))
        self.h = h
        self.info = self.stats()

    def step(self, t, sched=(2.0, 1.0, 81.0, 2.5)):
        self.ctx.check(self.ctx.L.he_lr_job_step(self.h, t, he_lr_sched(*sched)))

    def step_io(self, t, state_in, state_out, sched=(2.0, 1.0, 81.0, 2.5)):
        """One step with W, V loaded from / written to host words (numpy uint64)."""
        pin = None if state_in is None else state_in.ctypes.data_as(ctypes.c_void_p)
        pout = None if state_out is None else state_out.ctypes.data_as(ctypes.c_void_p)
        self.ctx.check(self.ctx.L.he_lr_job_step_io(self.h, t, he_lr_sched(*sched), pin, pout))

    def set_graph(self, on=True):
        self.ctx.check(self.ctx.L.he_lr_job_set_graph(self.h, int(on)))

    def set_refresh(self, boot=None):
        """Refresh W and V by bootstrapping with the parameters dict boot (slots,
        K, r, deg, scale_out, level_out), or by decryption and re-encryption (None)."""
        if boot is None:
            self.ctx.check(self.ctx.L.he_lr_job_set_refresh(self.h, None))
        else:
            p = he_boot_params(boot["slots"], boot["K"], boot["r"], boot["deg"], boot["scale_out"], boot["level_out"])
            self.ctx.check(self.ctx.L.he_lr_job_set_refresh(self.h, ctypes.byref(p)))

    def set_batch(self, blocks_per_launch):
        self.ctx.check(self.ctx.L.he_lr_job_set_batch(self.h, int(blocks_per_launch)))

    def weights(self, row=0):
        w = np.zeros(self.info.g)
        self.ctx.check(self.ctx.L.he_lr_job_weights(self.h, row, _ptr(w), len(w)))
        return w

    def all_weights(self):
        W, V = ctypes.c_void_p(), ctypes.c_void_p()
        self.ctx.check(self.ctx.L.he_lr_job_state(self.h, ctypes.byref(W), ctypes.byref(V)))
        return W, V

    def state_words(self):
        W, V = self.all_weights()
        out = []
        for h in (W, V):
            lv, sc = ctypes.c_int(), ctypes.c_double()
            self.ctx.check(self.ctx.L.he_ct_level(h, ctypes.byref(lv), ctypes.byref(sc)))
            w = np.zeros((2, lv.value + 1, self.ctx.n), np.uint64)
            self.ctx.check(self.ctx.L.he_ct_export(h, _ptr(w), w.size, None, None))
            out.append((w, lv.value, sc.value))
        return out

    def input(self, kind, index):
        o = ctypes.c_void_p()
        self.ctx.check(self.ctx.L.he_lr_job_input(self.h, kind, index, ctypes.byref(o)))
        return Ct(self.ctx, o)

    def block_grad(self, b):
        o = ctypes.c_void_p()
        self.ctx.check(self.ctx.L.he_lr_job_block_grad(self.h, b, ctypes.byref(o)))
        return Ct(self.ctx, o)

    def stats(self):
        s = he_lr_stats()
        self.ctx.check(self.ctx.L.he_lr_job_info(self.h, ctypes.byref(s)))
        return s

    def close(self):
        if getattr(self, "h", None):
            self.ctx.L.he_lr_job_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """he_lr_multi: several full-batch jobs stepped together (jobs stay owned by the caller)."""

    def __init__(self, ctx, jobs, blocks_per_launch=0):
        self.ctx, self.jobs = ctx, list(jobs)
        arr = (ctypes.c_void_p * len(jobs))(*[j.h.value for j in jobs])
        h = ctypes.c_void_p()
        ctx.check(ctx.L.he_lr_multi_create(ctx.h, arr, len(jobs), blocks_per_launch, ctypes.byref(h)))
        self.h = h

    def step(self, t, sched=(2.0, 1.0, 81.0, 2.5)):
        self.ctx.check(self.ctx.L.he_lr_multi_step(self.h, t, he_lr_sched(*sched)))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.L.he_lr_multi_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lr_iteration(ctx, Z, B, W, V, g, m, alpha, eta, inv_n, poly):
    arr = (ctypes.c_void_p * len(Z))(*[z.h.value for z in Z])
    p = np.asarray(poly, np.float64)
    Wo, Vo = ctypes.c_void_p(), ctypes.c_void_p()
    bh = B.h if B is not None else None  # None: the first-order baseline
    ctx.check(ctx.L.he_lr_iteration(ctx.h, arr, len(Z), bh, W.h, V.h, g, m, float(alpha), float(eta),
                                    float(inv_n), _ptr(p), ctypes.byref(Wo), ctypes.byref(Vo)))
    return Ct(ctx, Wo), Ct(ctx, Vo)


def lr_train(ctx, X, y, iters, sched=(2.0, 1.0, 81.0, 2.5), mode=FULL_BATCH, batch_rows=1024, poly=G8,
             enc_seed=3, key_seed=2, g=None):
    """he_lr_train: the whole training in one call; returns (decrypted weights
    of row 0 [g values], he_lr_stats)."""
    X = np.ascontiguousarray(X, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    n, f = X.shape
    if g is None:
        g = 1 << int(np.ceil(np.log2(f + 1)))
    w = np.zeros(g)
    st = he_lr_stats()
    ctx.check(ctx.L.he_lr_train(ctx.h, _ptr(X), _ptr(y), n, f, int(iters), he_lr_sched(*sched), mode, batch_rows,
                                poly, enc_seed, key_seed, _ptr(w), g, ctypes.byref(st)))
    return w, st


def launch_count():
    return int(load().he_launch_count())


def gauss_table(sigma):
    L = load()
    out = np.zeros(64, np.uint64)
    n = ctypes.c_size_t()
    rc = L.he_gauss_table(float(sigma), _ptr(out), 64, ctypes.byref(n))
    if rc:
        raise HeError(rc, "he_gauss_table")
    return out[:n.value]


def zeta_table(log_n):
    L = load()
    re = np.zeros(2 << log_n)
    im = np.zeros(2 << log_n)
    rc = L.he_zeta_table(log_n, _ptr(re), _ptr(im))
    if rc:
        raise HeError(rc, "he_zeta_table")
    return re, im


def lr_bbar_batches(ctx, X, y, batch_rows, g):
    """Bbar_k of every mini-batch, computed on the device: array [nbatch, g]."""
    X = np.ascontiguousarray(X, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    nb = -(-X.shape[0] // batch_rows)
    out = np.zeros((nb, g))
    ctx.check(ctx.L.he_lr_bbar_batches(ctx.h, _ptr(X), _ptr(y), X.shape[0], X.shape[1], batch_rows, g, _ptr(out)))
    return out


def lr_bbar(X, y, row0, rows, g):
    L = load()
    X = np.ascontiguousarray(X, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    out = np.zeros(g)
    rc = L.he_lr_bbar(_ptr(X), _ptr(y), X.shape[0], X.shape[1], row0, rows, g, _ptr(out))
    if rc:
        raise HeError(rc, "he_lr_bbar")
    return out
