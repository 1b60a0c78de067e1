"""The C-ABI library loads and exports every function include/ata.h declares
(no GPU work here)."""
import ctypes
import os
import re

import paper_1902_02104_gb300 as ata

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ata_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(ata.load()._name)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    lib = ata.load()
    assert lib.ata_status_string(0) == b"ATA_OK"
    assert lib.ata_status_string(7) == b"ATA_EBUSY"


def test_null_plan_rejected_without_device_work():
    lib = ata.load()
    assert lib.ata_execute(None, None, 1, None, None) == ata.ATA_EINVAL
    assert lib.ata_plan_workspace_size(None, None) == ata.ATA_EINVAL
    assert lib.ata_execute_batched(None, -1, None, None, None, None) == ata.ATA_EINVAL
    assert lib.ata_execute_batched(None, 0, None, None, None, None) == ata.ATA_OK
    assert lib.ata_gemm_tn(None, None, 1, None, 1, None, 1, None) == ata.ATA_EINVAL
    assert lib.ata_gemm_plan_create(None, 1, 1, 1, 0, None) == ata.ATA_EINVAL
    assert lib.ata_execute_host_async(None, None, 1, None) == ata.ATA_EINVAL
    assert lib.ata_plan_wait(None) == ata.ATA_EINVAL
    assert lib.ata_plan_graph_kernels(None, None) == ata.ATA_EINVAL
    assert lib.ata_batched_graph_kernels(None, -1, None, None) == ata.ATA_EINVAL
    assert lib.ata_server_kernels(None, None) == ata.ATA_EINVAL
    assert lib.ata_batch_create(None, None, 0, None, None, None) == ata.ATA_EINVAL
    assert lib.ata_batch_execute(None, None, None, None) == ata.ATA_EINVAL
    assert lib.ata_batch_graph_kernels(None, None) == ata.ATA_EINVAL
    lib.ata_batch_destroy(None)
    assert b"NULL" in lib.ata_last_error_message() or lib.ata_last_error_message() != b""


def test_server_argument_checks_without_device():
    lib = ata.load()
    h = ctypes.c_void_p()
    assert lib.ata_server_create(ctypes.byref(h), 0, 1, 4) == ata.ATA_EINVAL       # no budget
    assert lib.ata_server_create(ctypes.byref(h), 1 << 30, 1, 0) == ata.ATA_EINVAL  # no slots
    assert lib.ata_server_create(ctypes.byref(h), 1 << 30, 9, 4) == ata.ATA_EINVAL  # dtype
    t = ctypes.c_uint64()
    assert lib.ata_submit(None, 1, 1, None, 1, None, ctypes.byref(t)) == ata.ATA_EINVAL
    assert lib.ata_poll(None, 1, 0) == ata.ATA_EINVAL


def test_prepared_batch_argument_checks_without_device():
    lib = ata.load()
    h = ctypes.c_void_p()
    assert lib.ata_batch_create(ctypes.byref(h), None, -1, None, None, None) == ata.ATA_EINVAL
    assert lib.ata_batch_create(ctypes.byref(h), None, 2, None, None, None) == ata.ATA_EINVAL  # NULL arrays
    null_plans = (ctypes.c_void_p * 2)(None, None)
    z = (ctypes.c_int64 * 2)(1, 1)
    assert lib.ata_batch_create(ctypes.byref(h), null_plans, 2, z, z, z) == ata.ATA_EINVAL  # NULL plan
    assert not h.value
    # an empty batch is valid and queues nothing
    assert lib.ata_batch_create(ctypes.byref(h), None, 0, None, None, None) == ata.ATA_OK
    assert h.value
    assert lib.ata_batch_execute(h, None, None, None) == ata.ATA_OK
    k = ctypes.c_int32(-1)
    assert lib.ata_batch_graph_kernels(h, ctypes.byref(k)) == ata.ATA_OK and k.value == 0
    lib.ata_batch_destroy(h)
