"""The Fortran interface module (fortran/icon_dycore.f90) against the C header,
read as text: no Fortran compiler is installed on either machine this is
built and tested on, so the module's agreement with the ABI (Sec. 4.3: the
dycore is called from Fortran through iso_c_binding) is checked here.

* Every bind(c) derived type lists the fields of the C struct of the same name,
  in the same order and with the interoperable kind of each C type (for
  interoperable types that fixes the layout to C's; the C layout itself is
  checked against the ctypes mirrors in test_abi_layout.py).
* Every interface binds a function the header declares, with the same number
  of arguments and result kind, and passes each argument the way the C
  prototype takes it: a C scalar by value (the `value` attribute, same kind),
  a C `T**` as `type(c_ptr)` by reference, a pointer to one of the public
  structs as that derived type by reference, an opaque handle as
  `type(c_ptr), value`, a pointer to numbers or characters either by reference
  with the matching kind or as `type(c_ptr), value`."""
import os
import re

from c_harness import ROOT

HEADER = os.path.join(ROOT, "include", "icon_dycore.h")
MODULE = os.path.join(ROOT, "fortran", "icon_dycore.f90")
STRUCTS = ("icon_grid_desc_t", "icon_dycore_params_t", "icon_state_t")
C_KIND = {"int32_t": "c_int32_t", "int": "c_int", "double": "c_double", "float": "c_float",
          "int64_t": "c_int64_t", "char": "c_char"}


def _c_source():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    return re.sub(r"//[^\n]*", " ", src)


def _c_struct_fields():
    """{typedef name: [(field, c type), ...]} of the public structs."""
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s+\w+\s*\{(.*?)\}\s*(\w+)\s*;", _c_source(), flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(?:const\s+)?([\w]+(?:\s*\*+)?)\s*(.*)$", decl)
            base = m.group(1).replace(" ", "")
            for nm in m.group(2).split(","):
                nm = nm.strip()
                stars = len(nm) - len(nm.lstrip("*"))
                fields.append((nm.lstrip("*"), base + "*" * stars))
        out[name] = fields
    return out


def _c_prototypes():
    """{function: (result type, [parameter types])}."""
    out = {}
    for ret, name, params in re.findall(r"([\w\s\*]+?)\s*\b(icon_\w+)\s*\(([^;{}]*)\)\s*;", _c_source()):
        params = " ".join(params.split())
        plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        out[name] = (" ".join(ret.split()), plist)
    return out


def _c_param_class(p):
    """('scalar', kind) | ('ptrptr', base) | ('ptr', base) for a C parameter declaration."""
    p = re.sub(r"\bconst\b", "", p)
    stars = p.count("*")
    base = p.replace("*", " ").split()[0]
    if stars == 0:
        return "scalar", base
    return ("ptrptr" if stars >= 2 else "ptr"), base


def _fortran_lines():
    text = open(MODULE).read()
    text = re.sub(r"!.*", "", text)
    return [ln.strip() for ln in text.replace("&\n", " ").splitlines() if ln.strip()]


def _fortran_types():
    out, cur = {}, None
    for ln in _fortran_lines():
        m = re.match(r"type\s*,\s*bind\(c\)\s*,\s*public\s*::\s*(\w+)", ln, flags=re.I)
        if m:
            cur = out.setdefault(m.group(1), [])
            continue
        if cur is not None and re.match(r"end\s+type", ln, flags=re.I):
            cur = None
            continue
        if cur is not None:
            decl, names = ln.split("::")
            kind = re.search(r"\((\w+)\)", decl).group(1)
            cur += [(n.strip(), kind) for n in names.split(",")]
    return out


def _fortran_interfaces():
    """{bound C name: (result kind or None, [(arg, decl type, value?, array?)])}."""
    out, cur, args, decls, result = {}, None, None, None, None
    for ln in _fortran_lines():
        m = re.match(r"(?:(\w+\(\w+\))\s+)?(function|subroutine)\s+(\w+)\s*\(([^)]*)\)\s*bind\(c\s*,\s*name\s*=\s*\"(\w+)\"\)",
                     ln, flags=re.I)
        if m:
            result = re.search(r"\((\w+)\)", m.group(1)).group(1) if m.group(1) else None
            cur, decls = m.group(5), {}
            args = [a.strip() for a in m.group(4).split(",") if a.strip()]
            continue
        if cur and re.match(r"end\s+(function|subroutine)", ln, flags=re.I):
            out[cur] = (result, [(a,) + decls[a] for a in args])
            cur = None
            continue
        if cur and "::" in ln and not ln.lower().startswith("import"):
            decl, names = ln.split("::")
            kind = re.search(r"\((?:kind\s*=\s*)?(\w+)\)", decl).group(1)
            value = bool(re.search(r"\bvalue\b", decl, flags=re.I))
            for n in re.findall(r"(\w+)(\([^)]*\))?", names):
                array = bool(n[1]) or "dimension" in decl.lower()
                decls[n[0]] = (kind, value, array)
    return out


def test_bind_c_types_mirror_the_header_structs():
    c, f = _c_struct_fields(), _fortran_types()
    assert set(f) == set(STRUCTS)
    for name in STRUCTS:
        cf, ff = c[name], f[name]
        assert [n for n, _ in cf] == [n for n, _ in ff], name
        for (n, ct), (_, fk) in zip(cf, ff):
            want = "c_ptr" if "*" in ct else C_KIND[ct]
            assert fk == want, (name, n, ct, fk)


def test_interfaces_pass_arguments_the_way_the_prototypes_take_them():
    protos, ifaces = _c_prototypes(), _fortran_interfaces()
    assert len(ifaces) >= 15
    opaque = {"icon_grid_t", "icon_dycore_t", "icon_mlp_t"}
    for cname, (fres, fargs) in ifaces.items():
        assert cname in protos, cname
        cres, cparams = protos[cname]
        assert len(fargs) == len(cparams), cname
        if fres is None:
            assert cres == "void", cname
        elif fres == "c_ptr":
            assert "*" in cres, cname
        else:
            assert fres == C_KIND[cres], (cname, cres, fres)
        for (arg, kind, value, array), cp in zip(fargs, cparams):
            cls, base = _c_param_class(cp)
            where = (cname, arg, cp)
            if cls == "scalar":
                assert value and kind == C_KIND[base], where
            elif cls == "ptrptr":
                assert kind == "c_ptr" and not value, where
            elif base in STRUCTS:
                assert kind == base and not value and not array, where
            elif base in opaque:
                assert kind == "c_ptr" and value, where
            else:
                assert (kind == "c_ptr" and value) or (not value and kind == C_KIND[base]), where


def test_example_uses_only_routines_the_module_exports():
    src = re.sub(r"!.*", "", open(os.path.join(ROOT, "fortran", "example_step.f90")).read())
    public = set()
    for ln in _fortran_lines():
        if ln.lower().startswith("public ::"):
            public |= {n.strip() for n in ln.split("::")[1].split(",")}
    used = set(re.findall(r"\b(icon_\w+)\s*\(", src)) - set(STRUCTS)
    assert used and used <= public, used - public
