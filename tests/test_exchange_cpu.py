"""Host side of the rotation-sharded registration (no GPU): the merges of the
shard exchanges (csrc/exchange.h, compiled with g++), and the library's
all-gather callback driven over gloo by two ranks."""
import ctypes
import os
import socket
import subprocess

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exchange_merges(tmp_path):
    exe = str(tmp_path / "exchange_test")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_00115_b300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "exchange_test.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2502_00115_b300 import capi, shard

    cb = shard.allgather_callback()
    got = []
    # the library calls the callback with 4, 8 k and sizeof(dses_result) bytes
    for nbytes in (4, 8 * 16, ctypes.sizeof(capi.dses_result)):
        send = bytes((rank * 31 + i) % 251 for i in range(nbytes))
        sbuf = ctypes.create_string_buffer(send, nbytes)
        rbuf = ctypes.create_string_buffer(world * nbytes)
        rc = cb(None, ctypes.addressof(sbuf), nbytes, ctypes.addressof(rbuf))
        got.append((rc, rbuf.raw))
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_allgather_callback_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        for (rc, raw), nbytes in zip(out[r], (4, 128, len(out[r][2][1]) // world)):
            assert rc == 0
            want = b"".join(bytes((k * 31 + i) % 251 for i in range(nbytes)) for k in range(world))
            assert raw == want
