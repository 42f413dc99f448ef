"""placeholder"""
class TorError(Exception): pass
Context = TorResult = None
def tor_create(*a, **k): raise NotImplementedError
tor_destroy = tor_eval = tor_eval_batch = tor_submit = tor_poll = tor_strerror = load_library = library_path = tor_create
