"""Exported assets on disk: the mesh-UV carrier with its BVH (exm_mesh_export / _import), the
UV maps and optionally an environment map, as raw little-endian sections after a one-line
JSON header.  The serving registry reloads assets from these files without building their BVH
again.  This module moves bytes between files and the library; it does no arithmetic.

File layout: the JSON header (utf-8, one line, ending in a newline) gives, per section, its
name, dtype, shape, byte offset (from the end of the header line) and byte count.
"""
from __future__ import annotations

import json

import numpy as np
import torch

from . import native as N

SECTION_NAMES = ["V", "F", "UV", "Fuv", "bvh_nodes", "bvh_tris", "bvh_sphere"]
_NUMPY = {"float32": np.float32, "int32": np.int32, "uint8": np.uint8, "bfloat16": np.uint16, "float16": np.float16}


def export_mesh(mesh):
    """(AssetInfo, [numpy sections]) of a library mesh."""
    info = N.exm_mesh_export_info(mesh)
    secs = [np.empty(int(info.bytes[k]), np.uint8) for k in range(N.ASSET_SECTIONS)]
    N.exm_mesh_export(mesh, secs)
    return info, secs


def import_mesh(ctx, info, secs):
    """A library mesh from exported sections (checked by the library before use)."""
    return N.exm_mesh_import(ctx, info, [np.ascontiguousarray(s) for s in secs])


def save_asset(path, mesh, maps, env=None):
    """Writes mesh + BVH, maps [H, W, 8] (FP32/BF16/FP16 tensor) and an optional env [H, W, 3]."""
    info, secs = export_mesh(mesh)
    entries, blobs, off = [], [], 0

    def add(name, arr, dtype, shape):
        nonlocal off
        b = np.ascontiguousarray(arr).view(np.uint8).ravel()
        entries.append({"name": name, "dtype": dtype, "shape": list(shape), "offset": off, "bytes": int(b.size)})
        blobs.append(b)
        off += int(b.size)

    for k, name in enumerate(SECTION_NAMES):
        add(name, secs[k], "uint8", [secs[k].size])
    for name, t in (("maps", maps), ("env", env)):
        if t is None:
            continue
        t = t.detach().cpu().contiguous()
        dt = {torch.float32: "float32", torch.bfloat16: "bfloat16", torch.float16: "float16"}[t.dtype]
        arr = t.view(torch.int16).numpy().view(np.uint16) if dt == "bfloat16" else t.numpy()
        add(name, arr, dt, t.shape)
    header = {"format": "exmesh-asset", "version": int(info.version), "node_bytes": int(info.node_bytes),
              "nv": int(info.nv), "nf": int(info.nf), "nuv": int(info.nuv), "n_nodes": int(info.n_nodes),
              "endianness": "little", "sections": entries}
    with open(path, "wb") as f:
        f.write((json.dumps(header) + "\n").encode())
        for b in blobs:
            f.write(b.tobytes())


def read_asset(path):
    """(header, {name: numpy array}) of an asset file."""
    with open(path, "rb") as f:
        header = json.loads(f.readline().decode())
        base = f.tell()
        data = f.read()
    if header.get("format") != "exmesh-asset":
        raise ValueError(f"{path}: not an exmesh asset")
    out = {}
    for e in header["sections"]:
        raw = np.frombuffer(data, np.uint8, count=e["bytes"], offset=e["offset"])
        out[e["name"]] = raw.view(_NUMPY[e["dtype"]]).reshape(e["shape"]) if e["dtype"] != "uint8" else raw.copy()
    return header, out


def load_asset(path, ctx, device=0):
    """(mesh handle, maps tensor, env tensor or None) from an asset file, on `device`."""
    header, sec = read_asset(path)
    info = N.AssetInfo()
    info.version = header["version"]
    info.node_bytes = header["node_bytes"]
    info.nv, info.nf, info.nuv, info.n_nodes = header["nv"], header["nf"], header["nuv"], header["n_nodes"]
    for k, name in enumerate(SECTION_NAMES):
        info.bytes[k] = sec[name].size
    mesh = import_mesh(ctx, info, [sec[n] for n in SECTION_NAMES])
    dev = torch.device("cuda", device)
    tensors = []
    for name in ("maps", "env"):
        if name not in sec:
            tensors.append(None)
            continue
        e = next(x for x in header["sections"] if x["name"] == name)
        a = sec[name]
        t = torch.from_numpy(a.view(np.int16).copy()).view(torch.bfloat16) if e["dtype"] == "bfloat16" \
            else torch.from_numpy(a.copy())
        tensors.append(t.to(dev))
    return mesh, tensors[0], tensors[1]
