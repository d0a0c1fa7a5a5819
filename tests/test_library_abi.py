"""The C-ABI library builds, loads and exports every function include/ils.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(ils_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g
    from paper_2203_15340_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ils_setup", "ils_solve", "ils_solve_many", "ils_destroy", "ils_options_default",
                     "ils_status_string", "ils_refactor", "ils_refactor_async", "ils_setup_csr", "ils_batch_capture", "ils_batch_run"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header(libpath):
    from paper_2203_15340_gb300 import binding
    assert set(declared_functions()) <= set(binding.SIGNATURES)


def test_host_only_calls_without_gpu(libpath):
    from paper_2203_15340_gb300 import binding
    o = binding.options()
    assert o.max_outer == 20000 and abs(o.theta - 0.1) < 1e-15 and o.method == 0
    assert binding.status_string(2).startswith("A^T J A")
    lib = binding.lib()
    h = ctypes.c_void_p()
    # Invalid sizes are rejected on the host before any CUDA call.
    assert lib.ils_setup(ctypes.byref(h), 10, 5, 3, 7, 1, 10, None, None) == binding.ILS_ERR_INVALID_ARG
    assert lib.ils_setup(ctypes.byref(h), 10, 5, 8, 2, 0, 10, None, None) == binding.ILS_ERR_INVALID_ARG
    assert lib.ils_setup(ctypes.byref(h), 10, 5, 8, 2, 1, 9, None, None) == binding.ILS_ERR_INVALID_ARG
    assert lib.ils_options_default(None) == binding.ILS_ERR_INVALID_ARG


def test_csr_setup_rejections_without_gpu(libpath):
    """ils_setup_csr refuses bad sizes and unsupported option mixes before any CUDA call."""
    from paper_2203_15340_gb300 import binding
    lib = binding.lib()
    h = ctypes.c_void_p()
    fake = 256  # never dereferenced: every case below fails host-side validation first
    bad = binding.ILS_ERR_INVALID_ARG
    assert lib.ils_setup_csr(ctypes.byref(h), 10, 5, 3, 7, 20, fake, fake, fake, None, None) == bad  # p < n
    assert lib.ils_setup_csr(ctypes.byref(h), 10, 5, 8, 2, -1, fake, fake, fake, None, None) == bad  # nnz < 0
    assert lib.ils_setup_csr(ctypes.byref(h), 10, 5, 8, 2, 20, None, fake, fake, None, None) == bad  # no rowptr
    assert lib.ils_setup_csr(None, 10, 5, 8, 2, 20, fake, fake, fake, None, None) == bad
    for kw in (dict(route=binding.ILS_ROUTE_MATRIX_FREE),
               dict(method=binding.ILS_SP_RK_RGS, precision=binding.ILS_BF16_REFINE),
               dict(method=binding.ILS_SP_SCD, precision=binding.ILS_FP32_REFINE)):
        o = binding.options(**kw)
        assert lib.ils_setup_csr(ctypes.byref(h), 10, 5, 8, 2, 20, fake, fake, fake, ctypes.byref(o), None) == bad
    assert not h.value


def test_null_handles_are_rejected_on_the_host(libpath):
    """Every call that takes a handle refuses a null one before any CUDA call, and the
    destroy calls accept null (the header's error contract; runs without a GPU)."""
    from paper_2203_15340_gb300 import binding
    lib = binding.lib()
    bad = binding.ILS_ERR_INVALID_ARG
    fake = 256  # never dereferenced
    assert lib.ils_refactor(None, fake, 10, None) == bad
    assert lib.ils_refactor_async(None, fake, 10, None) == bad
    assert lib.ils_solve(None, fake, fake, 1, 1e-10, None, None) == bad
    assert lib.ils_solve_many(None, 1, fake, 10, fake, 10, 1, 1e-10, None, None) == bad
    assert lib.ils_get_matrix(None, 0, fake, 10, None) == bad
    assert lib.ils_aq_product(None, fake, fake, 0, None) == bad
    out = (ctypes.c_double * 7)()
    assert lib.ils_get_timings(None, out, 7) == -1
    assert lib.ils_batch_solve(None, 1, None, None, None, None, 1, 1e-10, None, None) == bad
    assert lib.ils_batch_capture(None, 0, 1, None, None, None, None, 1, 1e-10, 4, None) == bad
    assert lib.ils_batch_run(None, None, None) == bad
    assert lib.ils_batch_setup(None, 1, None, None, None) == bad
    b = ctypes.c_void_p()
    assert lib.ils_batch_setup(ctypes.byref(b), 0, None, None, None) == bad and not b.value
    assert lib.ils_mlp_create(None, 16, 256, 256, 0, None) == bad
    m = ctypes.c_void_p()
    assert lib.ils_mlp_create(ctypes.byref(m), 0, 256, 256, 0, None) == bad and not m.value
    assert lib.ils_mlp_num_params(None) == -1
    assert lib.ils_mlp_get_params(None, fake, None) == bad
    assert lib.ils_mlp_set_params(None, fake, None) == bad
    assert lib.ils_mlp_forward(None, 1, fake, fake, 256, 1, None) == bad
    assert lib.ils_solve_param(None, None, 1, fake, fake, 10, fake, 10, 1e-10, None, None) == bad
    lib.ils_destroy(None)
    lib.ils_batch_destroy(None)
    lib.ils_mlp_destroy(None)


def test_noalloc_cuda_failure_is_described_without_gpu(libpath):
    """With no CUDA device the no-allocation Gram fails its device lookup on the host: it
    returns ILS_ERR_CUDA and ils_last_error describes the failing call.  (Only where no
    device is visible: the pointers below are placeholders that are never dereferenced
    because the lookup fails first.)"""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is visible: the placeholder pointers must not reach a kernel")
    from paper_2203_15340_gb300 import binding
    lib = binding.lib()
    code = lib.ils_gram_noalloc(16, 8, 256, 16, 512, 8, None)
    assert code == binding.ILS_ERR_CUDA
    msg = lib.ils_last_error().decode()
    assert "ils_gram_noalloc" in msg and len(msg) > len("ils_gram_noalloc")


def test_new_options_are_validated_on_the_host(libpath):
    """Out-of-range values of the options added for the stop rules, the samplers and the
    estimates are rejected by ils_setup before any CUDA call."""
    from paper_2203_15340_gb300 import binding
    lib = binding.lib()
    h = ctypes.c_void_p()
    o = binding.options()
    assert o.stop_rule == 0 and o.estimate == 0 and o.alpha_mode == 0 and o.sampler == 0 and o.factor64 == 0
    assert o.theta_decay == 1.0 and o.theta_min == 0.0
    for field, bad in (("stop_rule", 3), ("alpha_mode", 2), ("sampler", 2), ("inner_form", 2),
                       ("wait_limit_ns", -1), ("lanczos_steps", 300), ("estimate", 3), ("theta_decay", 1.5),
                       ("theta_decay", -0.1), ("theta_min", -1e-3)):
        o = binding.options(**{field: bad})
        assert lib.ils_setup(ctypes.byref(h), 30, 5, 20, 10, 1, 30, ctypes.byref(o), None) == \
            binding.ILS_ERR_INVALID_ARG, field
    for kw in (dict(method=2, alpha_mode=1, alpha_fixed=0), dict(method=2, alpha_mode=1, alpha_fixed=6),
               dict(method=0, inner_form=1), dict(method=0, sampler=1)):
        o = binding.options(**kw)
        assert lib.ils_setup(ctypes.byref(h), 30, 5, 20, 10, 1, 30, ctypes.byref(o), None) == \
            binding.ILS_ERR_INVALID_ARG, kw
    assert lib.ils_set_wait_limit(None, 0) == binding.ILS_ERR_INVALID_ARG
    assert lib.ils_record_picks(None, None, 0) == binding.ILS_ERR_INVALID_ARG
    assert lib.ils_set_warmstart(None, None) == binding.ILS_ERR_INVALID_ARG
